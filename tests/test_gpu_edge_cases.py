"""Degenerate cases of the method against the oracle: a one-cell periodic mesh (the cell is its
own neighbour on both axes), a family of one member (the standalone method), the smallest
second-order member (E = 2, the two-stage midpoint method), and a mesh whose finest level is a
single 2 x 2 block of cells."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.dgsem import DGSEM
from oracle.perk import element_methods, max_wave_speed_dt, perk2_family, prkm_step
from oracle.treemesh import TreeMesh
from perk_inputs import isentropic_vortex, kelvin_helmholtz, nodal_state, refine_cells, uniform_cells
from tests.gpu_common import X3, solver_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_05144_gb300.build import build
    build()


def compare(cells, x0, L, ic, E, flux, steps, cfl=0.4, S=None):
    m = TreeMesh(cells, x0, L)
    U0 = nodal_state(ic, cells, x0, L, X3)
    fam = perk2_family(E, S)
    meth = element_methods(m.cells[:, 0], fam.R)
    dt = max_wave_speed_dt(U0, m.h, 3, cfl)
    s = solver_for(cells, x0, L, flux)
    s.set_perk2_disk(E, S)
    U = torch.from_numpy(U0.copy()).cuda()
    want = U0
    dg = DGSEM(m, 3, flux)
    for _ in range(steps):
        s.step(U, dt)
        want = prkm_step(dg.rhs, want, dt, fam, meth)
    s.check()
    return np.max(np.abs(U.cpu().numpy() - want)) / np.max(np.abs(want))


def test_one_cell_periodic_mesh():
    assert compare([(0, 0, 0)], -1.0, 2.0, kelvin_helmholtz, [4, 8], "hllc", 3) < 1e-12


def test_one_member_family_is_the_standalone_method():
    assert compare(uniform_cells(2), -1.0, 2.0, kelvin_helmholtz, [6], "hll", 3) < 1e-12


def test_smallest_member_two_stages():
    assert compare(uniform_cells(2), -1.0, 2.0, kelvin_helmholtz, [2], "hllc", 3, cfl=0.2) < 1e-12


def test_finest_level_is_one_block():
    # one level-2 cell of a level-1 mesh refined once: four fine cells and their hanging faces
    cells = refine_cells(uniform_cells(1), lambda l, ix, iy: (ix, iy) == (0, 0))
    assert compare(cells, -10.0, 20.0, isentropic_vortex, [2, 4], "hll", 3, S=4) < 1e-12
