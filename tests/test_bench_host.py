"""CPU checks of bench.py's host-side measurement helpers: the cell averages of a nodal state and
the coarse-against-fine L1 error behind the total-error comparison."""
import numpy as np
import pytest

bench = pytest.importorskip("bench")

from oracle.lgl import lgl_nodes_weights
from perk_inputs import kh_band_cells, uniform_cells


def test_cell_means_integrate_polynomials_exactly():
    # the 4-node Gauss-Lobatto rule is exact to degree 5 in each direction: over the reference
    # square the average of a + b x + c y + x^2 y^3 is a (odd moments vanish), that of x^2 y^2 is 1/9
    x, w = lgl_nodes_weights(3)
    X, Y = np.meshgrid(x, x, indexing="xy")   # [j, i]: node (i, j) at (x_i, y_j)
    U = np.zeros((2, 4, 4, 4))
    U[0, 0] = 2.0 + 0.5 * X - 0.25 * Y + X ** 2 * Y ** 3
    U[1, 0] = X ** 2 * Y ** 2
    U[:, 1] = 1.0
    m = bench.cell_means(U, w)
    np.testing.assert_allclose(m[:, 0], [2.0, 1.0 / 9.0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(m[:, 1], 1.0, rtol=0, atol=1e-15)


def test_l1_against_fine_aggregates_blocks():
    # a level-5 reference grid whose averages over the coarse leaves are reproduced exactly gives
    # zero; a leaf off by delta adds delta times its area (a fraction of the domain)
    ref_level = 5
    side = 1 << ref_level
    rng = np.random.default_rng(3)
    ref = rng.normal(size=(side, side))
    cells = np.asarray(kh_band_cells(2, 5, 0.1))
    means = np.array([ref[iy << (ref_level - l):(iy + 1) << (ref_level - l),
                          ix << (ref_level - l):(ix + 1) << (ref_level - l)].mean() for l, ix, iy in cells])
    assert bench.l1_against_fine(cells, means, ref, ref_level) == pytest.approx(0.0, abs=1e-14)
    k = int(np.argmin(cells[:, 0]))
    bumped = means.copy()
    bumped[k] += 0.3
    area = 1.0 / (1 << (2 * int(cells[k, 0])))
    assert bench.l1_against_fine(cells, bumped, ref, ref_level) == pytest.approx(0.3 * area, rel=1e-12)
    # a uniform mesh at the reference level compares cell by cell
    fine = uniform_cells(ref_level)
    vals = np.array([ref[iy, ix] for _, ix, iy in fine])
    assert bench.l1_against_fine(fine, vals + 1.0, ref, ref_level) == pytest.approx(1.0, rel=1e-12)
