"""Accuracy of the partitioned step against the standalone method (the comparison of Sec. 5):
the isentropic vortex on the two-level mesh, one period (t = 20), P-ERK2 {4, 8} against the
8-stage member alone at the same dt, both measured against the exact translated vortex."""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.lgl import lgl_nodes_weights
from perk_inputs import isentropic_vortex, nodal_state, vortex_two_level_cells

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2403_05144_gb300.build import build
    build()


def density_errors(cells, U, exact, L):
    _, w = lgl_nodes_weights(3)
    e = np.abs(U[:, 0] - exact[:, 0])
    h = L / 2.0 ** np.asarray(cells)[:, 0]
    l1 = np.sum((0.5 * h) ** 2 * np.einsum("eji,j,i->e", e, w, w)) / (L * L)
    return l1, e.max()


def run_vortex(E, t_end, cfl):
    from paper_2403_05144_gb300 import PerkSolver
    cells = vortex_two_level_cells()
    x, _ = lgl_nodes_weights(3)
    s = PerkSolver(surface_flux="hll")
    s.upload_mesh(cells, -10.0, 20.0)
    s.set_perk2_disk(E, 8)
    U = torch.from_numpy(nodal_state(isentropic_vortex, cells, -10.0, 20.0, x)).cuda()
    dt = s.compute_dt(U, cfl)
    n = math.ceil(t_end / dt)
    for _ in range(n):
        s.step(U, t_end / n)
    s.check()
    exact = nodal_state(isentropic_vortex, cells, -10.0, 20.0, x, t=t_end)
    return density_errors(cells, U.cpu().numpy(), exact, 20.0)


def test_vortex_partitioned_error_within_a_quarter_of_the_standalone_error():
    l1_p, li_p = run_vortex([4, 8], 20.0, 0.5)
    l1_f, li_f = run_vortex([8], 20.0, 0.5)
    assert l1_p <= 1.25 * l1_f, (l1_p, l1_f)
    assert li_p <= 1.25 * li_f, (li_p, li_f)
    # and both are the spatial error of a smooth solution, not an instability
    assert l1_f < 1e-3 and li_f < 5e-2
