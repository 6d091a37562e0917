"""GPU parity of the HLLE surface flux and of the subcell shock capturing (blended volume term)
with the oracle (oracle/euler.py hlle_flux, oracle/shock.py)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.dgsem import DGSEM
from oracle.perk import element_methods, max_wave_speed_dt, perk2_family, prkm_step
from oracle.shock import ShockCapturingDGSEM, blending_factor
from oracle.treemesh import TreeMesh
from perk_inputs import kelvin_helmholtz, kh_band_cells, nodal_state
from tests.gpu_common import X3, discontinuous_state, rel_err_per_var

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_05144_gb300.build import build
    build()


def solver(cells, shock, E=None, equations="euler", mu=0.0):
    from paper_2403_05144_gb300 import PerkSolver
    s = PerkSolver(surface_flux="hlle", shock_capturing=shock, equations=equations, mu=mu)
    s.upload_mesh(cells, -1.0, 2.0)
    if E is not None:
        s.set_perk2_disk(E)
    return s


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_hlle_rhs():
    cells = kh_band_cells(4, 6, 0.05)
    U = discontinuous_state(cells, -1.0, 2.0)
    got = solver(cells, None).rhs_full(cuda(U)).cpu().numpy()
    want = DGSEM(TreeMesh(cells, -1.0, 2.0), 3, "hlle").rhs(U)
    assert rel_err_per_var(got, want) < 1e-12


@pytest.mark.parametrize("variable,jump", [("density_pressure", 0.05), ("density", 0.2)])
def test_shock_capturing_rhs(variable, jump):
    # a state with jumps at every node: elements blend, some reach the cap (and with the
    # smaller jump some stay unblended)
    cells = kh_band_cells(4, 6, 0.05)
    U = discontinuous_state(cells, -1.0, 2.0, jump=jump)
    alpha = blending_factor(U, X3, variable=variable)
    assert np.any(alpha == 0.5) and np.any((alpha > 0) & (alpha < 0.5))
    got = solver(cells, variable).rhs_full(cuda(U)).cpu().numpy()
    want = ShockCapturingDGSEM(TreeMesh(cells, -1.0, 2.0), 3, "hlle", variable=variable).rhs(U)
    assert rel_err_per_var(got, want) < 1e-12


def test_shock_capturing_active_stages_and_steps():
    cells = kh_band_cells(4, 6, 0.05)
    m = TreeMesh(cells, -1.0, 2.0)
    E = [4, 6, 10, 16]
    fam = perk2_family(E)
    meth = element_methods(m.cells[:, 0], fam.R)
    U = discontinuous_state(cells, -1.0, 2.0, jump=0.2)
    sc = ShockCapturingDGSEM(m, 3, "hlle", variable="density")
    full = sc.rhs(U)
    s = solver(cells, "density", E)
    for i in (0, 8, 15):
        active = np.array([fam.active(int(r), i) for r in meth])
        got = s.rhs_active(i, cuda(U), out=cuda(np.full_like(U, 7.0))).cpu().numpy()
        assert np.all(got[~active] == 7.0)
        assert rel_err_per_var(got[active], full[active]) < 1e-12
    # three steps from the Kelvin-Helmholtz state
    U0 = nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3)
    dt = max_wave_speed_dt(U0, m.h, 3, 0.5)
    Ug = cuda(U0)
    want = U0
    for _ in range(3):
        s.step(Ug, dt)
        want = prkm_step(sc.rhs, want, dt, fam, meth)
    s.check()
    assert np.max(np.abs(Ug.cpu().numpy() - want)) / np.max(np.abs(want)) < 1e-11


def test_shock_capturing_with_navier_stokes():
    from oracle.shock import ShockCapturingNavierStokesDGSEM
    cells = kh_band_cells(3, 5, 0.05)
    U = discontinuous_state(cells, -1.0, 2.0, jump=0.05)
    o = ShockCapturingNavierStokesDGSEM(TreeMesh(cells, -1.0, 2.0), 3, "hlle", mu=1e-3)
    got = solver(cells, "density_pressure", equations="navier_stokes", mu=1e-3).rhs_full(cuda(U)).cpu().numpy()
    assert rel_err_per_var(got, o.rhs(U)) < 1e-12


def test_derivatives_are_refused_with_shock_capturing():
    from paper_2403_05144_gb300 import PerkError
    cells = kh_band_cells(3, 5, 0.05)
    U = cuda(discontinuous_state(cells, -1.0, 2.0))
    s = solver(cells, "density", [4, 8])
    with pytest.raises(PerkError):
        s.rhs_jvp(U, U)
    with pytest.raises(PerkError):
        s.step_vjp(U, 1e-4, U.clone())
