"""Pins of the oracle's DGSEM right-hand side on periodic quadtrees: mesh
counts, free-stream preservation at hanging faces, discrete conservation,
entropy conservation of the flux-differencing volume term and the RHS
consistency order."""
import numpy as np
import pytest

from oracle import euler
from oracle.dgsem import DGSEM
from oracle.lgl import lgl_nodes_weights
from oracle.treemesh import TreeMesh, is_balanced
from perk_inputs import (isentropic_vortex, kh_band_cells, nodal_state, prim_to_cons, smooth_random_state,
                         uniform_cells, vortex_two_level_cells)

X3, W3 = lgl_nodes_weights(3)


@pytest.fixture(scope="module")
def vortex_mesh():
    return TreeMesh(vortex_two_level_cells(), -10.0, 20.0)


def test_vortex_mesh_counts(vortex_mesh):
    # 16x16 base with the central 8x8 block refined: 192 + 256 cells, 32 hanging faces
    m = vortex_mesh
    assert m.n_elem == 448
    assert len(m.conforming) == 848
    assert len(m.hanging) == 64          # two half-face records per hanging face
    assert is_balanced(m)


def test_kh_band_mesh_balanced():
    m = TreeMesh(kh_band_cells(4, 7), -1.0, 2.0)
    assert is_balanced(m)
    assert set(np.unique(m.cells[:, 0]).tolist()) == {4, 5, 6, 7}


@pytest.mark.parametrize("flux", ["hll", "hllc"])
def test_free_stream_preservation(vortex_mesh, flux):
    U = nodal_state(lambda X, Y: prim_to_cons(1.2 + 0 * X, 0.3 + 0 * X, -0.4 + 0 * X, 0.9 + 0 * X),
                    vortex_mesh.cells, -10.0, 20.0, X3)
    K = DGSEM(vortex_mesh, 3, flux).rhs(U)
    assert np.max(np.abs(K)) < 1e-12


def discontinuous_state(cells, x0, L, seed=7):
    U = smooth_random_state(cells, x0, L, X3, seed=seed, amplitude=0.2)
    return U * (1.0 + 0.05 * np.random.default_rng(seed).uniform(-1, 1, size=U.shape))


@pytest.mark.parametrize("flux", ["hll", "hllc", "ec"])
def test_discrete_conservation_nonconforming(vortex_mesh, flux):
    U = discontinuous_state(vortex_mesh.cells, -10.0, 20.0)
    dg = DGSEM(vortex_mesh, 3, flux)
    K = dg.rhs(U)
    scale = np.max(np.abs(K)) * 20.0 ** 2
    assert np.all(np.abs(dg.integrate(K)) < 1e-13 * scale)


def test_entropy_conservation_conforming():
    # EC volume flux + EC surface flux on a conforming periodic mesh: no entropy production
    cells = uniform_cells(3)
    m = TreeMesh(cells, 0.0, 1.0)
    U = discontinuous_state(cells, 0.0, 1.0)
    W = euler.entropy_variables(np.moveaxis(U, 1, 0))
    for flux, sign in (("ec", 0), ("hll", -1), ("hllc", -1)):
        K = DGSEM(m, 3, flux).rhs(U)
        ds = np.einsum("e,veji,veji,ji->", (0.5 * m.h) ** 2, W, np.moveaxis(K, 1, 0), np.outer(W3, W3))
        if sign == 0:
            assert abs(ds) < 1e-13 * np.max(np.abs(K))
        else:
            assert ds < -1e-4                   # the upwind surface fluxes dissipate entropy


def test_rhs_consistency_order():
    # F(u_exact) -> du/dt of the translating vortex at rate ~N (= 3) on two-level meshes
    errs = []
    for lev in (4, 5):
        cells = vortex_two_level_cells(lev, 2 ** (lev - 2), 3 * 2 ** (lev - 2))
        m = TreeMesh(cells, -10.0, 20.0)
        U = nodal_state(isentropic_vortex, cells, -10.0, 20.0, X3)
        eps = 1e-6
        Ut = (nodal_state(isentropic_vortex, cells, -10.0, 20.0, X3, t=eps)
              - nodal_state(isentropic_vortex, cells, -10.0, 20.0, X3, t=-eps)) / (2 * eps)
        K = DGSEM(m, 3, "hll").rhs(U)
        errs.append(np.sqrt(np.einsum("e,evji,ji->", (0.5 * m.h) ** 2, (K - Ut) ** 2, np.outer(W3, W3))))
    assert np.log2(errs[0] / errs[1]) > 2.7


def test_mortar_side_symmetry(vortex_mesh):
    # mirroring the mesh and state in x maps the RHS onto its mirror image
    cells = np.array(vortex_mesh.cells)
    n = 1 << cells[:, 0]
    mirrored = np.stack([cells[:, 0], n - 1 - cells[:, 1], cells[:, 2]], axis=1)
    U = discontinuous_state(vortex_mesh.cells, -10.0, 20.0)
    Um = U[:, :, :, ::-1].copy()
    Um[:, 1] *= -1.0
    K = DGSEM(vortex_mesh, 3, "hll").rhs(U)
    Km = DGSEM(TreeMesh(mirrored, -10.0, 20.0), 3, "hll").rhs(Um)
    Kback = Km[:, :, :, ::-1].copy()
    Kback[:, 1] *= -1.0
    np.testing.assert_allclose(Kback, K, atol=1e-12 * np.max(np.abs(K)))
