"""Pins of the oracle's dense P-ERK step on the 2D DGSEM: conservation with
shared weights, reduction to the single-member method, member assignment by
level and second-order temporal convergence."""
import numpy as np
import pytest

from oracle.dgsem import DGSEM
from oracle.lgl import lgl_nodes_weights
from oracle.perk import element_methods, max_wave_speed_dt, perk2_family, prkm_step, rk_step
from oracle.treemesh import TreeMesh
from perk_inputs import isentropic_vortex, nodal_state, prim_to_cons, smooth_random_state, uniform_cells, \
    vortex_two_level_cells

X3, _ = lgl_nodes_weights(3)


def test_member_assignment_by_level():
    # finest level -> member R-1, next -> R-2, all coarser levels -> member 0
    levels = np.array([4, 5, 6, 7, 7, 3])
    np.testing.assert_array_equal(element_methods(levels, 3), [0, 0, 1, 2, 2, 0])
    np.testing.assert_array_equal(element_methods(levels, 4), [0, 1, 2, 3, 3, 0])
    # fewer levels than members: the coarse members stay unused
    np.testing.assert_array_equal(element_methods(np.array([5, 6, 7]), 4), [1, 2, 3])


def test_step_conserves_on_two_level_mesh():
    cells = vortex_two_level_cells(3, 2, 6)
    m = TreeMesh(cells, -10.0, 20.0)
    dg = DGSEM(m, 3, "hll")
    U = smooth_random_state(cells, -10.0, 20.0, X3, amplitude=0.2)
    fam = perk2_family([4, 8])
    meth = element_methods(m.cells[:, 0], fam.R)
    assert set(meth.tolist()) == {0, 1}
    U1 = prkm_step(dg.rhs, U, 0.2, fam, meth)
    np.testing.assert_allclose(dg.integrate(U1), dg.integrate(U), rtol=1e-14, atol=1e-13)


def test_single_level_reduces_to_standalone_method():
    cells = uniform_cells(2)
    m = TreeMesh(cells, 0.0, 1.0)
    dg = DGSEM(m, 3, "hll")
    U = smooth_random_state(cells, 0.0, 1.0, X3, amplitude=0.2)
    fam = perk2_family([4, 8])
    meth = element_methods(m.cells[:, 0], fam.R)
    assert np.all(meth == 1)
    alone = perk2_family([8])
    np.testing.assert_array_equal(prkm_step(dg.rhs, U, 0.01, fam, meth), rk_step(dg.rhs, U, 0.01, alone.A[0], alone.b))


def test_second_order_in_time_two_levels():
    cells = vortex_two_level_cells(3, 2, 6)
    m = TreeMesh(cells, -10.0, 20.0)
    dg = DGSEM(m, 3, "hll")
    U0 = nodal_state(isentropic_vortex, cells, -10.0, 20.0, X3)
    fam = perk2_family([4, 8])
    meth = element_methods(m.cells[:, 0], fam.R)
    T = 0.8

    def run(n):
        U = U0
        for _ in range(n):
            U = prkm_step(dg.rhs, U, T / n, fam, meth)
        return U

    ref = run(32)
    errs = [np.max(np.abs(run(n) - ref)) for n in (4, 8)]
    assert np.log2(errs[0] / errs[1]) > 1.8


def test_cfl_step_free_stream():
    cells = vortex_two_level_cells()
    m = TreeMesh(cells, -10.0, 20.0)
    U = nodal_state(lambda X, Y: prim_to_cons(1.0 + 0 * X, 0.5 + 0 * X, -0.25 + 0 * X, 1.0 / 1.4 + 0 * X),
                    cells, -10.0, 20.0, X3)
    # c = 1, lambda = 0.5 + 0.25 + 2; finest h = 20/32
    assert max_wave_speed_dt(U, m.h, 3, 0.8) == pytest.approx(0.8 * (20 / 32) / (4 * 2.75), rel=1e-14)
