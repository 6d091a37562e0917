"""GPU parity of the Navier-Stokes (BR1) path with the oracle: full and
partitioned right-hand sides and P-ERK steps on meshes with hanging faces."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.br1 import NavierStokesDGSEM
from oracle.perk import element_methods, max_wave_speed_dt, perk2_family, prkm_step
from oracle.treemesh import TreeMesh
from perk_inputs import kh_band_cells, nodal_state, shear_layer, vortex_two_level_cells
from tests.gpu_common import X3, discontinuous_state, rel_err_per_var

pytestmark = pytest.mark.gpu
MU = 2e-3


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_05144_gb300.build import build
    build()


def ns_solver(cells, flux="hll", E=None, mu=MU):
    from paper_2403_05144_gb300 import PerkSolver
    s = PerkSolver(surface_flux=flux, equations="navier_stokes", mu=mu, prandtl=0.72)
    s.upload_mesh(cells, 0.0, 1.0)
    if E:
        s.set_perk2_disk(E)
    return s


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("flux", ["hll", "hllc"])
@pytest.mark.parametrize("cells_fn", [lambda: vortex_two_level_cells(3, 2, 6), lambda: kh_band_cells(3, 5, 0.05)])
def test_rhs_full(flux, cells_fn):
    cells = cells_fn()
    U = discontinuous_state(cells, 0.0, 1.0)
    got = ns_solver(cells, flux).rhs_full(cuda(U)).cpu().numpy()
    want = NavierStokesDGSEM(TreeMesh(cells, 0.0, 1.0), 3, flux, mu=MU).rhs(U)
    assert rel_err_per_var(got, want) < 1e-12


def test_rhs_active_every_stage():
    cells = kh_band_cells(3, 5, 0.05)
    U = discontinuous_state(cells, 0.0, 1.0)
    E = [4, 8, 16]
    s = ns_solver(cells, "hll", E)
    m = TreeMesh(cells, 0.0, 1.0)
    fam = perk2_family(E)
    meth = element_methods(m.cells[:, 0], fam.R)
    full = NavierStokesDGSEM(m, 3, "hll", mu=MU).rhs(U)
    for i in range(fam.S):
        active = np.array([fam.active(int(r), i) for r in meth])
        got = s.rhs_active(i, cuda(U), out=cuda(np.full_like(U, 7.0))).cpu().numpy()
        assert np.all(got[~active] == 7.0)
        assert rel_err_per_var(got[active], full[active]) < 1e-12


def test_shear_layer_steps():
    cells = kh_band_cells(3, 5, 0.05)
    U0 = nodal_state(shear_layer, cells, 0.0, 1.0, X3)
    m = TreeMesh(cells, 0.0, 1.0)
    E = [4, 8, 16]
    fam = perk2_family(E)
    dt = max_wave_speed_dt(U0, m.h, 3, 0.5)
    s = ns_solver(cells, "hll", E, mu=4e-4)
    U = cuda(U0.copy())
    for _ in range(5):
        s.step(U, dt)
    s.check()
    ns = NavierStokesDGSEM(m, 3, "hll", mu=4e-4)
    want = U0
    for _ in range(5):
        want = prkm_step(ns.rhs, want, dt, fam, element_methods(m.cells[:, 0], fam.R))
    assert np.max(np.abs(U.cpu().numpy() - want)) / np.max(np.abs(want)) < 1e-11


def oracle_tableau_into(solver, fam):
    """Hand the oracle's coefficient table to the library (order, E, c, a_{i,i-1})."""
    S = fam.S
    a = np.zeros((fam.R, S))
    for r in range(fam.R):
        for i in range(2, S):
            a[r, i] = fam.A[r][i, i - 1]
    solver.set_tableau(fam.order, fam.E, fam.c, a)


@pytest.mark.parametrize("equations", ["euler", "navier_stokes"])
def test_third_order_steps(equations):
    from oracle.dgsem import DGSEM
    from oracle.perk import perk3_family
    from paper_2403_05144_gb300 import PerkSolver
    cells = kh_band_cells(3, 5, 0.05)
    m = TreeMesh(cells, 0.0, 1.0)
    U0 = nodal_state(shear_layer, cells, 0.0, 1.0, X3)
    fam = perk3_family([4, 8, 16])
    dt = max_wave_speed_dt(U0, m.h, 3, 0.5)
    s = PerkSolver(surface_flux="hll", equations=equations, mu=4e-4 if equations != "euler" else 0.0)
    s.upload_mesh(cells, 0.0, 1.0)
    oracle_tableau_into(s, fam)
    U = cuda(U0.copy())
    for _ in range(3):
        s.step(U, dt)
    s.check()
    rhs = (NavierStokesDGSEM(m, 3, "hll", mu=4e-4) if equations != "euler" else DGSEM(m, 3, "hll")).rhs
    want = U0
    for _ in range(3):
        want = prkm_step(rhs, want, dt, fam, element_methods(m.cells[:, 0], fam.R))
    assert np.max(np.abs(U.cpu().numpy() - want)) / np.max(np.abs(want)) < 1e-11


@pytest.mark.parametrize("use_graph", [True, False])
def test_inviscid_terms_in_one_launch_bitwise_equal(use_graph):
    # one launch for a stage's inviscid face and volume terms (then BR1's launches) against two:
    # the same arithmetic, so the same bits; a one-launch step mode falls back for Navier-Stokes
    from paper_2403_05144_gb300 import PerkSolver
    cells = kh_band_cells(3, 5, 0.05)
    U0 = cuda(nodal_state(shear_layer, cells, 0.0, 1.0, X3))
    out = []
    for mode in (1, 2, 0):
        s = PerkSolver(surface_flux="hll", equations="navier_stokes", mu=MU, prandtl=0.72, use_graph=use_graph)
        s.set_stage_fusion(mode)
        s.upload_mesh(cells, 0.0, 1.0)
        s.set_perk2_disk([4, 8, 16])
        U = U0.clone()
        dt = s.compute_dt(U, 0.5)
        for _ in range(3):
            s.step(U, dt)
        s.check()
        out.append(U)
    assert torch.equal(out[0], out[2]) and torch.equal(out[1], out[2])
    acc = None
    s = PerkSolver(surface_flux="hll", equations="navier_stokes", mu=MU, prandtl=0.72)
    s.upload_mesh(cells, 0.0, 1.0)
    s.set_perk2_disk([4, 8, 16])
    acc = s.step_profiled(U0.clone(), 1e-4, acc)
    assert acc.launches[0] == 0 and acc.launches[1] == 16 and acc.launches[3] == 16
