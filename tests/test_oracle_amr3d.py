"""Pins of the 3D AMR oracle (enstrophy indicator of the paper's Eq. Enstrophy, octree balance,
exact transfer): closed-form enstrophy of polynomial velocity fields, the sibling and 2:1 rules,
refine-then-coarsen identity, conservation and polynomial exactness of the transfer."""
import math

import numpy as np
import pytest

from oracle.amr3d import adapt3, balance3, desired_levels3, enstrophy_indicator, new_cells3, transfer3
from oracle.dgsem3d import DGSEM3D
from oracle.lgl import lgl_nodes_weights
from oracle.octree import OctreeMesh, is_balanced3
from perk_inputs.octree import (block_refined_cells3, node_coordinates3, nodal_state3, prim_to_cons3,
                                smooth_random_state3, taylor_green, uniform_cells3)

L = 2.0


def _mesh(cells):
    return OctreeMesh(np.asarray(cells), 0.0, L)


@pytest.mark.parametrize("N", [2, 3])
def test_enstrophy_of_a_polynomial_velocity_in_closed_form(N):
    a, b, c, d = 0.7, -0.4, 0.9, 0.3
    cells = block_refined_cells3(2, 1, 3)
    x, _ = lgl_nodes_weights(N)
    X, Y, Z = node_coordinates3(cells, 0.0, L, x)
    rho = 1.2
    U = prim_to_cons3(rho * np.ones_like(X), a * Y + b * Z * Z, c * X * Z, d * X * Y, np.ones_like(X))
    U = np.moveaxis(U, 0, 1)
    # curl v = (d x - c x, 2 b z - d y, c z - a)
    w = (d * X - c * X, 2 * b * Z - d * Y, c * Z - a)
    want = (0.5 * rho * (w[0] ** 2 + w[1] ** 2 + w[2] ** 2)).reshape(len(cells), -1).max(axis=1)
    got = enstrophy_indicator(U, _mesh(cells).h, N)
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(want)


def test_taylor_green_enstrophy_maximum_converges():
    """The TGV vorticity's largest |omega|^2 is 4 (omega_z = 2 sin x sin y cos z at a node of both
    meshes): the indicator's maximum approaches 0.5 * 4 at the rate of the N = 2 derivative."""
    errs = []
    for level in (2, 3):
        cells = uniform_cells3(level)
        x, _ = lgl_nodes_weights(2)
        U = nodal_state3(taylor_green, cells, 0.0, 2 * math.pi, x)
        eta = enstrophy_indicator(U, OctreeMesh(np.asarray(cells), 0.0, 2 * math.pi).h, 2)
        errs.append(abs(eta.max() - 2.0))
    assert errs[1] < errs[0] / 3.0 and errs[1] < 0.25


def test_siblings_coarsen_only_together():
    mesh = _mesh(uniform_cells3(1))
    assert np.all(balance3(mesh, np.zeros(8, dtype=int)) == 0)
    d = np.zeros(8, dtype=int)
    d[3] = 1
    assert np.all(balance3(mesh, d) == 1)


def test_balance_propagates_and_the_new_mesh_is_balanced():
    mesh = _mesh(uniform_cells3(2))
    d = np.full(mesh.n_elem, 1)                  # everything wants to coarsen ...
    d[5] = 3                                     # ... except one cell, which refines
    out = balance3(mesh, d)
    assert out[5] == 3 and np.all(out >= d)
    # the refined cell's face neighbours stay at level 2, and so do their whole sibling groups
    for (A, B, _) in mesh.conforming:
        if 5 in (A, B):
            assert out[B if A == 5 else A] >= 2
    cells = new_cells3(mesh, out)
    new = _mesh(cells)
    assert is_balanced3(new)
    # a coarsened parent replaces exactly eight old cells
    lev = mesh.cells[:, 0]
    assert len(cells) == int(np.sum(out > lev) * 8 + np.sum(out == lev) + np.sum(out < lev) // 8)


def test_refine_then_coarsen_is_the_identity():
    cells = block_refined_cells3(2, 1, 3)
    mesh = _mesh(cells)
    x, _ = lgl_nodes_weights(2)
    U = smooth_random_state3(cells, 0.0, L, x, amplitude=0.2)
    U *= 1.0 + 0.05 * np.random.default_rng(4).uniform(-1, 1, U.shape)
    fine, Uf, _ = adapt3(mesh, U, 0, 10, 0, 0, desired=mesh.cells[:, 0] + 1)
    back, Ub, _ = adapt3(fine, Uf, 0, 10, 0, 0, desired=fine.cells[:, 0] - 1)
    assert [tuple(c) for c in back.cells.tolist()] == [tuple(c) for c in mesh.cells.tolist()]
    assert np.max(np.abs(Ub - U)) < 1e-13 * np.max(np.abs(U))


def test_coarsening_conserves_and_is_exact_on_polynomials():
    cells = uniform_cells3(2)
    mesh = _mesh(cells)
    N = 2
    x, _ = lgl_nodes_weights(N)
    U = smooth_random_state3(cells, 0.0, L, x, amplitude=0.2)
    U *= 1.0 + 0.05 * np.random.default_rng(5).uniform(-1, 1, U.shape)
    coarse, Uc, _ = adapt3(mesh, U, 0, 10, 0, 0, desired=mesh.cells[:, 0] - 1)
    assert coarse.n_elem == 8
    I0 = DGSEM3D(mesh, N).integrate(U)
    I1 = DGSEM3D(coarse, N).integrate(Uc)
    assert np.max(np.abs(I1 - I0)) < 1e-13 * np.max(np.abs(I0))
    # a polynomial of degree N on each coarse cell survives refine + coarsen and coarsen alone
    ccells = uniform_cells3(1)
    Xc, Yc, Zc = node_coordinates3(ccells, 0.0, L, x)
    Xf, Yf, Zf = node_coordinates3(cells, 0.0, L, x)

    def poly(X, Y, Z):
        return np.stack([1 + 0.1 * X * Y, 0.2 * Z * Z, X - Y, 0.3 * X * Z, 3 + Y * Y])

    Ufine = np.moveaxis(poly(Xf, Yf, Zf), 0, 1)
    _, Up, _ = adapt3(mesh, Ufine, 0, 10, 0, 0, desired=mesh.cells[:, 0] - 1)
    assert np.max(np.abs(Up - np.moveaxis(poly(Xc, Yc, Zc), 0, 1))) < 1e-13


def test_transfer_of_a_refined_polynomial_is_exact():
    cells = uniform_cells3(1)
    x, _ = lgl_nodes_weights(3)
    X, Y, Z = node_coordinates3(cells, 0.0, L, x)
    U = np.moveaxis(np.stack([X ** 3, Y * Z, Z ** 2 * X, np.ones_like(X), X * Y * Z]), 0, 1)
    fine = new_cells3(_mesh(cells), np.ones(8, dtype=int) * 2)
    Uf = transfer3(cells, U, fine, N=3)
    Xf, Yf, Zf = node_coordinates3(fine, 0.0, L, x)
    want = np.moveaxis(np.stack([Xf ** 3, Yf * Zf, Zf ** 2 * Xf, np.ones_like(Xf), Xf * Yf * Zf]), 0, 1)
    assert np.max(np.abs(Uf - want)) < 1e-13


def test_desired_levels_thresholds():
    cells = uniform_cells3(2)
    mesh = _mesh(cells)
    eta = np.zeros(mesh.n_elem)
    eta[0] = 5.0
    d = desired_levels3(mesh, eta, 1, 3, refine_above=1.0, coarsen_below=0.5)
    assert d[0] == 3 and is_balanced3(_mesh(new_cells3(mesh, d)))


def test_taylor_green_bench_mesh_recipe():
    """The benchmark's 3D mesh: 16^3 cells adapted twice by the enstrophy indicator (levels 4-6,
    refine above 1.2, coarsen below 0.3) has 30,080 cells (3,136 / 4,928 / 22,016 on levels
    4 / 5 / 6), and a third cycle leaves it unchanged."""
    x, _ = lgl_nodes_weights(2)
    cells = uniform_cells3(4)
    U = nodal_state3(taylor_green, cells, 0.0, 2 * math.pi, x)
    m = OctreeMesh(np.asarray(cells), 0.0, 2 * math.pi)
    for _ in range(2):
        m, U, _ = adapt3(m, U, 4, 6, 1.2, 0.3)
    assert m.n_elem == 30080
    assert np.bincount(m.cells[:, 0]).tolist()[4:] == [3136, 4928, 22016]
    m3, _, d = adapt3(m, U, 4, 6, 1.2, 0.3)
    assert np.array_equal(d, m.cells[:, 0])
