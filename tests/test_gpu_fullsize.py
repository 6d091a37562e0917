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
    # The right-hand side is a sum of derivative terms of size up to (2/h) |f(u)|.  In this
    # low-Mach state they cancel almost completely: the pressure (~7.9) has no gradient at t = 0
    # and the density RHS vanishes analytically (rho = 1, v_x depends on y only, v_y on x only),
    # so what remains (momentum RHS <= 5, density RHS ~1e-13) is far below the terms whose
    # rounding it carries (~1e-11 absolute).  Errors are therefore measured against the scale of
    # the derivative terms, (2/h_min) max |u|; a wrong term would be 1e-3 of that, not 1e-12.
    scale = (2.0 / m.h.min()) * np.max(np.abs(U))
    for i in (0, 9, 15):
        active = np.array([fam.active(int(r), i) for r in meth])
        got = s.rhs_active(i, torch.from_numpy(U).cuda(),
                           out=torch.from_numpy(np.full_like(U, 7.0)).cuda()).cpu().numpy()
        assert np.all(got[~active] == 7.0)
        assert np.max(np.abs(got[active] - full[active])) / scale < 1e-12, i
        # and against the RHS itself where it is not a cancellation remainder (energy)
        assert np.max(np.abs(got[active][:, 3] - full[active][:, 3])) / np.max(np.abs(full[:, 3])) < 1e-10
