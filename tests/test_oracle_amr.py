"""Pins of the oracle's AMR: indicator closed form, balance and sibling rules,
exact transfer (refine then coarsen is the identity) and conservation."""
import numpy as np
import pytest

from oracle.amr import adapt, balance, desired_levels, indicator, new_cells, transfer
from oracle.dgsem import DGSEM
from oracle.lgl import lgl_nodes_weights
from oracle.treemesh import TreeMesh, is_balanced
from perk_inputs import kelvin_helmholtz, kh_band_cells, nodal_state, smooth_random_state, uniform_cells, \
    vortex_two_level_cells

X3, W3 = lgl_nodes_weights(3)


def test_indicator_linear_density_closed_form():
    # rho = a + b x on [0, 1]^2 with 4x4 cells: eta = h b / rho_mean(cell)
    cells = uniform_cells(2)
    a, b = 2.0, 0.5
    U = nodal_state(lambda X, Y: np.stack([a + b * X, 0 * X, 0 * X, 2.5 + 0 * X]), cells, 0.0, 1.0, X3)
    eta = indicator(U)
    h = 0.25
    xc = (np.array([c[1] for c in cells]) + 0.5) * h
    np.testing.assert_allclose(eta, h * b / (a + b * xc), rtol=1e-13)


def test_lohner_indicator_hand_computed_values():
    # v_x on every row of the element: (1, 1, 3, 1) at the four x nodes; rho = 2.
    # Triples along x: (1, 1, 3): |3 - 2 + 1| / (2 + 0 + 0.2 (3 + 2 + 1)) = 2 / 3.2;
    # (1, 3, 1): |1 - 6 + 1| / (2 + 2 + 0.2 (1 + 6 + 1)) = 4 / 5.6.  Along y every
    # column is constant: 0.  Largest: 4 / 5.6.
    from oracle.amr import indicator, lohner_indicator
    row = np.array([1.0, 1.0, 3.0, 1.0])
    vx = np.tile(row, (4, 1))[None]                        # [1, j, i]
    U = np.zeros((1, 4, 4, 4))
    U[:, 0] = 2.0
    U[:, 1] = 2.0 * vx
    U[:, 3] = 5.0
    assert abs(indicator(U, kind="lohner_vx")[0] - 4.0 / 5.6) < 1e-15
    # the same pattern along y gives the same value; constants give 0; scale-free
    assert abs(lohner_indicator(np.swapaxes(vx, 1, 2))[0] - 4.0 / 5.6) < 1e-15
    assert lohner_indicator(np.full((1, 4, 4), 3.7))[0] == 0.0
    assert abs(lohner_indicator(-7.5 * vx)[0] - 4.0 / 5.6) < 1e-15
    # a resolved tanh layer scores lower than the same layer on a four times coarser cell
    x = np.array([-1.0, -np.sqrt(0.2), np.sqrt(0.2), 1.0])
    fine = np.tanh(0.5 * x)[None, None, :].repeat(4, axis=1)
    coarse = np.tanh(2.0 * x)[None, None, :].repeat(4, axis=1)
    assert lohner_indicator(fine)[0] < lohner_indicator(coarse)[0]


def test_single_flag_propagates_for_balance():
    # refining one fine cell next to a coarse neighbour forces the neighbour to refine
    cells = vortex_two_level_cells(3, 2, 6)             # levels 3 and 4
    m = TreeMesh(cells, 0.0, 1.0)
    d = m.cells[:, 0].copy()
    target = next(e for e, c in enumerate(cells) if c == (4, 4, 4))   # a fine cell on the block edge
    d[target] = 5
    d = balance(m, d)
    new = TreeMesh(new_cells(m, d), 0.0, 1.0)
    assert is_balanced(new)
    assert any(c[0] == 5 for c in new.cells.tolist())
    # its level-3 neighbour across x (cell (3, 1, 2)) had to refine to level 4
    e = next(e for e, c in enumerate(cells) if c == (3, 1, 2))
    assert d[e] == 4


def test_coarsening_needs_all_siblings():
    cells = uniform_cells(2)
    m = TreeMesh(cells, 0.0, 1.0)
    d = m.cells[:, 0].copy()
    kids = [e for e, c in enumerate(cells) if c[1] // 2 == 0 and c[2] // 2 == 0]
    for e in kids[:3]:
        d[e] = 1
    assert np.all(balance(m, d)[kids] == 2)           # three of four: no coarsening
    d[kids[3]] = 1
    d2 = balance(m, d)
    assert np.all(d2[kids] == 1)
    assert len(new_cells(m, d2)) == 16 - 3


def test_refine_then_coarsen_is_identity_and_conservative():
    cells = vortex_two_level_cells(3, 2, 6)
    m = TreeMesh(cells, -1.0, 2.0)
    U = smooth_random_state(cells, -1.0, 2.0, X3, amplitude=0.3)
    # refine everything once, then coarsen back
    fine = new_cells(m, m.cells[:, 0] + 1)
    Uf = transfer([tuple(c) for c in cells], U, fine)
    mf = TreeMesh(fine, -1.0, 2.0)
    back = new_cells(mf, mf.cells[:, 0] - 1)
    assert back == [tuple(c) for c in TreeMesh(cells, -1, 2.0).cells.tolist()] or sorted(back) == sorted(cells)
    Ub = transfer([tuple(c) for c in fine], Uf, back)
    order = {c: e for e, c in enumerate(back)}
    Ub_orig = np.array([Ub[order[tuple(c)]] for c in cells])
    np.testing.assert_allclose(Ub_orig, U, atol=1e-13)
    np.testing.assert_allclose(DGSEM(mf, 3).integrate(Uf), DGSEM(m, 3).integrate(U), rtol=1e-14)


def test_coarsening_projection_conserves_discontinuous_data():
    cells = uniform_cells(3)
    m = TreeMesh(cells, 0.0, 1.0)
    U = smooth_random_state(cells, 0.0, 1.0, X3, amplitude=0.3)
    U = U * (1 + 0.1 * np.random.default_rng(2).uniform(-1, 1, U.shape))
    coarse = new_cells(m, m.cells[:, 0] - 1)
    Uc = transfer([tuple(c) for c in cells], U, coarse)
    np.testing.assert_allclose(DGSEM(TreeMesh(coarse, 0.0, 1.0), 3).integrate(Uc), DGSEM(m, 3).integrate(U),
                               rtol=1e-14)


def test_kh_adapt_cycle_balanced_and_bounded():
    cells = kh_band_cells(4, 6, 0.05)
    m = TreeMesh(cells, -1.0, 2.0)
    U = nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3)
    m2, U2, d = adapt(m, U, 4, 7, 0.1, 0.02)
    assert is_balanced(m2)
    assert m2.cells[:, 0].min() >= 4 and m2.cells[:, 0].max() <= 7
    assert m2.n_elem != m.n_elem
    np.testing.assert_allclose(DGSEM(m2, 3).integrate(U2), DGSEM(m, 3).integrate(U), rtol=1e-13)
