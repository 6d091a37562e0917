"""Parity at the benchmark's full sizes, in the launch configuration bench.py times (CUDA-graph
replay, default launch shapes): one P-ERK2 {4,6,10,16} step on the initially adapted
Kelvin-Helmholtz mesh (3,904 cells, levels 4-7) against the oracle's dense step, every output;
and the Navier-Stokes shear layer on its initially adapted three-level mesh (6,400 cells), the
partitioned right-hand side of three stages against the oracle's masked full one."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.amr import desired_levels, indicator, new_cells
from oracle.br1 import NavierStokesDGSEM
from oracle.dgsem import DGSEM
from oracle.perk import element_methods, perk2_family, prkm_step
from oracle.treemesh import TreeMesh
from perk_inputs import kelvin_helmholtz, nodal_state, shear_layer, uniform_cells
from tests.gpu_common import X3

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_05144_gb300.build import build
    build()


def initially_adapted(ic, base, x0, L, amr, kind, cycles):
    """The benchmark's initial mesh: adaptation cycles on the initial state itself."""
    cells = uniform_cells(base)
    for _ in range(cycles):
        m = TreeMesh(cells, x0, L)
        U = nodal_state(ic, cells, x0, L, X3)
        cells = new_cells(m, desired_levels(m, indicator(U, kind=kind), **amr))
    return cells


def test_kelvin_helmholtz_step_at_bench_size():
    from paper_2403_05144_gb300 import PerkSolver
    cells = initially_adapted(kelvin_helmholtz, 4, -1.0, 2.0,
                              dict(level_min=4, level_max=7, refine_above=0.1, coarsen_below=0.02), "density", 3)
    assert len(cells) == 3904
    U0 = nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3)
    E = [4, 6, 10, 16]
    s = PerkSolver(surface_flux="hllc", use_graph=True)
    s.upload_mesh(cells, -1.0, 2.0)
    s.set_perk2_disk(E)
    U = torch.from_numpy(U0.copy()).cuda()
    dt = s.compute_dt(U, 0.7)
    s.step(U, dt)
    s.check()
    m = TreeMesh(cells, -1.0, 2.0)
    fam = perk2_family(E)
    want = prkm_step(DGSEM(m, 3, "hllc").rhs, U0, dt, fam, element_methods(m.cells[:, 0], fam.R))
    got = U.cpu().numpy()
    # per-RHS differences of ~1e-13 pass through 16 stages (|dt lambda| up to ~30)
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < 1e-11


def test_shear_layer_partitioned_rhs_at_bench_size():
    from paper_2403_05144_gb300 import PerkSolver, perk3_disk_tableau
    cells = initially_adapted(shear_layer, 6, 0.0, 1.0,
                              dict(level_min=6, level_max=8, refine_above=0.1, coarsen_below=0.02), "lohner_vx", 2)
    assert len(cells) == 6400
    U = nodal_state(shear_layer, cells, 0.0, 1.0, X3)
    E = [4, 8, 16]
    s = PerkSolver(surface_flux="hll", equations="navier_stokes", mu=1.0 / 2500.0, prandtl=0.72)
    s.upload_mesh(cells, 0.0, 1.0)
    c, a = perk3_disk_tableau(E)
    s.set_tableau(3, E, c, a)
    m = TreeMesh(cells, 0.0, 1.0)
    fam = perk2_family(E)                    # the members' activity pattern is the same at third order
    meth = element_methods(m.cells[:, 0], fam.R)
    full = NavierStokesDGSEM(m, 3, "hll", mu=1.0 / 2500.0, prandtl=0.72).rhs(U)
    # the density right-hand side of this state vanishes analytically (rho = 1, v_x depends on y
    # only, v_y on x only): it is rounding noise of ~1e-13 on both sides, left by cancelling flux
    # terms as large as the momentum ones, so every variable is measured against the largest
    # variable's scale
    scale = np.max(np.abs(full))
    for i in (0, 9, 15):
        active = np.array([fam.active(int(r), i) for r in meth])
        got = s.rhs_active(i, torch.from_numpy(U).cuda(),
                           out=torch.from_numpy(np.full_like(U, 7.0)).cuda()).cpu().numpy()
        assert np.all(got[~active] == 7.0)
        for v in range(4):
            den = max(np.max(np.abs(full[active][:, v])), scale)
            assert np.max(np.abs(got[active][:, v] - full[active][:, v])) / den < 1e-12, (i, v)
