"""Pins of the 3D BR1 oracle (viscous terms of the paper's Taylor-Green run, Sec. 7.1.3): free
streams, exact reduction to the pinned 2D BR1 oracle on extruded meshes, axis relabelling,
conservation at hanging faces, and convergence to mu times the Laplacian of a shear wave and
kappa times the Laplacian of a temperature wave."""
import math

import numpy as np
import pytest

from oracle.br1 import NavierStokesDGSEM
from oracle.br1_3d import NavierStokesDGSEM3D
from oracle.lgl import lgl_nodes_weights
from oracle.octree import OctreeMesh
from oracle.treemesh import TreeMesh
from perk_inputs import smooth_random_state, vortex_two_level_cells
from perk_inputs.octree import (block_refined_cells3, extrude_cells, node_coordinates3, prim_to_cons3, refine_cells3,
                                smooth_random_state3, uniform_cells3)

L = 2.0
MU = 0.01


def _mesh(cells):
    return OctreeMesh(np.asarray(cells), -1.0, L)


def test_free_stream_has_no_viscous_terms():
    cells = block_refined_cells3(2, 1, 3)
    U = np.empty((len(cells), 5, 3, 3, 3))
    U[:] = prim_to_cons3(1.2, 0.3, -0.4, 0.5, 1.1)[None, :, None, None, None]
    K = NavierStokesDGSEM3D(_mesh(cells), 2, mu=MU).viscous_rhs(U)
    assert np.max(np.abs(K)) < 1e-13


def test_reduces_to_the_2d_br1_oracle_on_an_extruded_mesh():
    cells2 = vortex_two_level_cells(2, 1, 3)
    cells3 = extrude_cells(cells2)
    N = 3
    x, _ = lgl_nodes_weights(N)
    U2 = smooth_random_state(cells2, -1.0, L, x, amplitude=0.1)
    U2 *= 1.0 + 0.03 * np.random.default_rng(2).uniform(-1, 1, U2.shape)
    K2 = NavierStokesDGSEM(TreeMesh(np.asarray(cells2), -1.0, L), N, "hll", mu=MU).viscous_rhs(U2)
    index2 = {tuple(c): e for e, c in enumerate(cells2)}
    U3 = np.zeros((len(cells3), 5, N + 1, N + 1, N + 1))
    for e3, (l, ix, iy, iz) in enumerate(cells3):
        U3[e3, [0, 1, 2, 4]] = U2[index2[(l, ix, iy)]][:, None, :, :]
    K3 = NavierStokesDGSEM3D(_mesh(cells3), N, "hll", mu=MU).viscous_rhs(U3)
    scale = np.max(np.abs(K2))
    for e3, (l, ix, iy, iz) in enumerate(cells3):
        want = K2[index2[(l, ix, iy)]]
        assert np.max(np.abs(K3[e3, [0, 1, 2, 4]] - want[:, None, :, :])) < 1e-12 * scale
        assert np.max(np.abs(K3[e3, 3])) < 1e-12 * scale


def test_axis_relabelling():
    cells = refine_cells3(uniform_cells3(2), lambda l, ix, iy, iz: 1 <= ix < 2 and 0 <= iy < 3 and 2 <= iz < 4)
    x, _ = lgl_nodes_weights(2)
    U = smooth_random_state3(cells, -1.0, L, x, amplitude=0.1)
    U *= 1.0 + 0.03 * np.random.default_rng(3).uniform(-1, 1, U.shape)
    K = NavierStokesDGSEM3D(_mesh(cells), 2, mu=MU).viscous_rhs(U)
    cells_p = [(l, iy, iz, ix) for (l, ix, iy, iz) in cells]

    def relabel(A):
        return np.transpose(A, (0, 1, 4, 2, 3))[:, [0, 2, 3, 1, 4]]

    Kp = NavierStokesDGSEM3D(_mesh(cells_p), 2, mu=MU).viscous_rhs(relabel(U))
    assert np.max(np.abs(Kp - relabel(K))) < 1e-12 * np.max(np.abs(K))


@pytest.mark.parametrize("N", [2, 3])
def test_conservation_at_hanging_faces(N):
    cells = block_refined_cells3(2, 1, 3)
    mesh = _mesh(cells)
    x, _ = lgl_nodes_weights(N)
    U = smooth_random_state3(cells, -1.0, L, x, amplitude=0.1)
    U *= 1.0 + 0.03 * np.random.default_rng(4).uniform(-1, 1, U.shape)
    op = NavierStokesDGSEM3D(mesh, N, mu=MU)
    K = op.viscous_rhs(U)
    total = op.integrate(K)
    assert np.max(np.abs(total)) < 1e-13 * np.max(np.abs(K)) * L ** 3


def _wave_errors(kind):
    N = 3
    x, w = lgl_nodes_weights(N)
    errs = []
    for level in (1, 2, 3):
        cells = uniform_cells3(level)
        X, Y, Z = node_coordinates3(cells, -1.0, L, x)
        k = 2.0 * math.pi / L
        one = np.ones_like(X)
        if kind == "shear":
            U = np.moveaxis(prim_to_cons3(one, 0.1 * np.sin(k * Y), 0 * one, 0 * one, one), 0, 1)
            op = NavierStokesDGSEM3D(_mesh(cells), N, mu=MU)
            got = op.viscous_rhs(U)[:, 1]
            want = -MU * 0.1 * k * k * np.sin(k * Y)
        else:
            T = 1.0 + 0.1 * np.sin(k * Z)
            U = np.moveaxis(prim_to_cons3(one, 0 * one, 0 * one, 0 * one, T), 0, 1)      # rho = 1: p = T
            op = NavierStokesDGSEM3D(_mesh(cells), N, mu=MU)
            got = op.viscous_rhs(U)[:, 4]
            want = -op.kappa * 0.1 * k * k * np.sin(k * Z)
        mesh = _mesh(cells)
        errs.append(np.sqrt(np.einsum("e,ekji,k,j,i->", (0.5 * mesh.h) ** 3, (got - want) ** 2, w, w, w)))
    return errs


@pytest.mark.parametrize("kind", ["shear", "heat"])
def test_viscous_terms_converge_to_the_laplacian(kind):
    """mu d2v1/dy2 for a shear wave, kappa d2T/dz2 for a temperature wave at rest."""
    errs = _wave_errors(kind)
    assert errs[0] > errs[1] > errs[2]
    assert math.log2(errs[1] / errs[2]) > 1.5, errs
