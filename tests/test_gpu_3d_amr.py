"""GPU parity of the 3D AMR cycle (enstrophy indicator of the paper's Eq. Enstrophy, octree
balance, exact transfer) with the 3D oracle: indicator values, the library's own decisions and
the replayed oracle decisions, transferred states, and a dynamic P-ERK3 {3,4,6} run."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.amr3d import adapt3, balance3, desired_levels3, enstrophy_indicator, new_cells3, transfer3
from oracle.dgsem3d import DGSEM3D, max_wave_speed_dt3
from oracle.lgl import lgl_nodes_weights
from oracle.octree import OctreeMesh
from oracle.perk import element_methods, perk3_family, prkm_step
from perk_inputs.octree import (block_refined_cells3, nodal_state3, refine_cells3, smooth_random_state3,
                                taylor_green, uniform_cells3)

pytestmark = pytest.mark.gpu

L = 2.0 * math.pi


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_05144_gb300.build import build
    build()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def mesh_of(cells):
    return OctreeMesh(np.asarray(cells), 0.0, L)


def solver(cells, N=2):
    from paper_2403_05144_gb300.perk3d import Perk3DSolver
    s = Perk3DSolver(N=N, surface_flux="hlle")
    s.upload_mesh(cells, 0.0, L)
    return s


def three_level_cells():
    c = refine_cells3(uniform_cells3(2), lambda l, ix, iy, iz: 1 <= ix < 3 and 0 <= iy < 2 and 1 <= iz < 4)
    return refine_cells3(c, lambda l, ix, iy, iz: l == 3 and 3 <= ix < 5 and 1 <= iy < 3 and 3 <= iz < 5)


def robust_thresholds(eta, lo_q=0.3, hi_q=0.7):
    """Thresholds halfway between neighbouring distinct indicator values, so that no decision
    hangs on the last bits of a value."""
    v = np.unique(eta)
    i, j = int(lo_q * (len(v) - 1)), int(hi_q * (len(v) - 1))
    return 0.5 * (v[j] + v[j + 1]), 0.5 * (v[i] + v[i + 1])


@pytest.mark.parametrize("N", [2, 3])
def test_indicator_matches_oracle(N):
    cells = three_level_cells()
    x, _ = lgl_nodes_weights(N)
    U = nodal_state3(taylor_green, cells, 0.0, L, x)
    got = solver(cells, N).amr_indicator(cuda(U)).cpu().numpy()
    want = enstrophy_indicator(U, mesh_of(cells).h, N)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(want)


@pytest.mark.parametrize("N", [2, 3])
def test_replayed_decisions_give_the_oracle_mesh_and_state(N):
    cells = three_level_cells()
    m = mesh_of(cells)
    x, _ = lgl_nodes_weights(N)
    U = smooth_random_state3(cells, 0.0, L, x, amplitude=0.2)
    U *= 1.0 + 0.05 * np.random.default_rng(9).uniform(-1, 1, U.shape)
    rng = np.random.default_rng(10)
    lev = m.cells[:, 0]
    wish = lev + rng.integers(-1, 2, size=len(lev))
    d = balance3(m, np.clip(wish, 2, 4))
    s = solver(cells, N)
    Un = s.adapt(cuda(U), desired=d).cpu().numpy()
    want_cells = new_cells3(m, d)
    assert [tuple(c) for c in s.cells.tolist()] == [tuple(c) for c in want_cells]
    want = transfer3([tuple(c) for c in cells], U, want_cells, N)
    assert np.max(np.abs(Un - want)) <= 1e-13 * np.max(np.abs(want))


def test_own_decisions_match_the_oracle():
    cells = uniform_cells3(3)
    m = mesh_of(cells)
    x, _ = lgl_nodes_weights(2)
    U = nodal_state3(taylor_green, cells, 0.0, L, x)
    eta = enstrophy_indicator(U, m.h, 2)
    up, down = robust_thresholds(eta)
    s = solver(cells)
    Un = s.adapt(cuda(U), level_min=2, level_max=4, refine_above=up, coarsen_below=down)
    m2, U2, _ = adapt3(m, U, 2, 4, up, down)
    assert [tuple(c) for c in s.cells.tolist()] == [tuple(c) for c in m2.cells.tolist()]
    assert np.max(np.abs(Un.cpu().numpy() - U2)) <= 1e-13 * np.max(np.abs(U2))


def test_refine_then_coarsen_restores_the_state():
    cells = block_refined_cells3(2, 1, 3)
    x, _ = lgl_nodes_weights(2)
    U0 = smooth_random_state3(cells, 0.0, L, x, amplitude=0.2)
    s = solver(cells)
    lev = np.asarray(cells)[:, 0]
    U1 = s.adapt(cuda(U0), desired=lev + 1)
    U2 = s.adapt(U1, desired=np.asarray(s.cells)[:, 0] - 1)
    assert [tuple(c) for c in s.cells.tolist()] == [tuple(c) for c in cells]
    assert np.max(np.abs(U2.cpu().numpy() - U0)) <= 1e-13 * np.max(np.abs(U0))


def test_dynamic_perk3_run_with_replayed_decisions():
    """Taylor-Green from 4^3 cells, levels 2-4: two initial cycles, then six P-ERK3 {3,4,6}
    steps with an AMR cycle after every second step; the oracle's decisions are replayed."""
    cells = uniform_cells3(2)
    x, _ = lgl_nodes_weights(2)
    Uo = nodal_state3(taylor_green, cells, 0.0, L, x)
    m = mesh_of(cells)
    fam = perk3_family([3, 4, 6])
    a = np.zeros((fam.R, fam.S))
    for r in range(fam.R):
        for i in range(2, fam.S):
            a[r, i] = fam.A[r][i, i - 1]
    s = solver(cells)
    s.set_tableau(3, fam.E, fam.c, a)
    U = cuda(Uo)
    prm = dict(level_min=2, level_max=4)

    def cycle(m, Uo, U):
        eta = enstrophy_indicator(Uo, m.h, 2)
        up, down = robust_thresholds(eta, 0.4, 0.75)
        d = desired_levels3(m, eta, prm["level_min"], prm["level_max"], up, down)
        m2, Uo2, _ = adapt3(m, Uo, prm["level_min"], prm["level_max"], up, down, desired=d)
        U2 = s.adapt(U, desired=d)
        assert [tuple(c) for c in s.cells.tolist()] == [tuple(c) for c in m2.cells.tolist()]
        return m2, Uo2, U2

    for _ in range(2):
        m, Uo, U = cycle(m, Uo, U)
    assert len(set(m.cells[:, 0].tolist())) >= 2
    dt = max_wave_speed_dt3(Uo, m.h, 2, 0.5)
    for k in range(6):
        s.step(U, dt)
        Uo = prkm_step(DGSEM3D(m, 2, "hlle").rhs, Uo, dt, fam, element_methods(m.cells[:, 0], fam.R))
        if k % 2 == 1:
            m, Uo, U = cycle(m, Uo, U)
    s.check()
    got = U.cpu().numpy()
    assert np.max(np.abs(got - Uo)) <= 1e-11 * np.max(np.abs(Uo))
