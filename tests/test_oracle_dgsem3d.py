"""Pins of the 3D oracle (octree DGSEM of the paper's Sec. 7.1.3) against what the
mathematics fixes: mesh counts, free-stream preservation at hanging faces, discrete
conservation, entropy conservation of the EC scheme, exact reduction to the pinned
2D oracle for z-independent states, consistency order against an exact solution,
axis-permutation and mirror symmetry, the face L2 projection, and the 3D fluxes."""

import math

import numpy as np
import pytest

from oracle import euler, euler3d
from oracle.dgsem import DGSEM
from oracle.dgsem3d import DGSEM3D, face_l2_projection, max_wave_speed_dt3
from oracle.lgl import l2_project_two_halves, lgl_nodes_weights
from oracle.octree import OctreeMesh, is_balanced3
from oracle.perk import element_methods, perk3_family, prkm_step
from oracle.treemesh import TreeMesh
from perk_inputs import smooth_random_state, vortex_two_level_cells
from perk_inputs.octree import (block_refined_cells3, density_wave3, extrude_cells, nodal_state3, prim_to_cons3,
                                refine_cells3, slab_cells3, smooth_random_state3, uniform_cells3)

L = 2.0


def _mesh(cells, x0=-1.0, length=L):
    return OctreeMesh(np.asarray(cells), x0, length)


def test_block_mesh_counts():
    mesh = _mesh(block_refined_cells3(2, 1, 3))
    assert mesh.n_elem == 56 + 64
    # 4^3 base cells, 3 x 64 periodic base faces; per axis 4 between refined cells (-> 16 fine faces),
    # 8 between a refined and an unrefined cell (hanging: 4 small faces each), 52 between coarse ones;
    # each refined base cell adds 12 faces between its own children
    assert len(mesh.conforming) == 3 * 52 + 3 * 4 * 4 + 8 * 12
    assert len(mesh.hanging) == 3 * 8 * 4
    assert is_balanced3(mesh)


def test_slab_mesh_is_balanced_and_sized():
    cells = slab_cells3(2, 4, 1.0 / 16.0)
    mesh = _mesh(cells)
    assert is_balanced3(mesh)
    assert set(mesh.cells[:, 0]) == {2, 3, 4}


@pytest.mark.parametrize("flux", ["hll", "hllc", "hlle", "ec"])
def test_free_stream_preserved_at_hanging_faces(flux):
    mesh = _mesh(block_refined_cells3(2, 1, 3))
    op = DGSEM3D(mesh, 2, flux)
    n = 3
    U = np.empty((mesh.n_elem, 5, n, n, n))
    U[:] = prim_to_cons3(1.2, 0.3, -0.4, 0.5, 1.1)[None, :, None, None, None]
    K = op.rhs(U)
    assert np.max(np.abs(K)) < 1e-12


@pytest.mark.parametrize("N", [2, 3])
def test_discrete_conservation(N):
    mesh = _mesh(block_refined_cells3(2, 1, 3))
    op = DGSEM3D(mesh, N, "hllc")
    x, _ = lgl_nodes_weights(N)
    U = smooth_random_state3(mesh.cells, -1.0, L, x, amplitude=0.1)
    K = op.rhs(U)
    total = op.integrate(K)
    scale = np.max(np.abs(K)) * L ** 3
    assert np.max(np.abs(total)) < 1e-13 * scale


def test_entropy_conservation_of_ec_scheme_and_dissipation_of_hll():
    mesh = _mesh(uniform_cells3(1))
    x, w = lgl_nodes_weights(3)
    U = smooth_random_state3(mesh.cells, -1.0, L, x, amplitude=0.2)
    # nodal noise on the density makes the traces jump across faces (sampled smooth data would not)
    U[:, 0] *= 1.0 + 0.05 * np.random.default_rng(3).uniform(-1.0, 1.0, U[:, 0].shape)
    W = np.einsum("k,j,i->kji", w, w, w)
    ent = {}
    for flux in ("ec", "hll", "hlle"):
        K = DGSEM3D(mesh, 3, flux).rhs(U)
        wv = euler3d.entropy_variables(np.moveaxis(U, 1, 0))
        ent[flux] = np.einsum("e,vekji,evkji,kji->", (0.5 * mesh.h) ** 3, wv, K, W)
        ent[flux + "_scale"] = np.einsum("e,vekji,evkji,kji->", (0.5 * mesh.h) ** 3, np.abs(wv), np.abs(K), W)
    assert abs(ent["ec"]) < 1e-13 * ent["ec_scale"]
    assert ent["hll"] < -1e-8 * ent["hll_scale"]
    assert ent["hlle"] < -1e-8 * ent["hlle_scale"]


@pytest.mark.parametrize("flux", ["hll", "hllc", "hlle"])
def test_reduces_to_the_2d_oracle_on_an_extruded_mesh(flux):
    """A z-independent state with v3 = 0 on an octree extruded from a quadtree: every x-y
    plane of nodes carries the 2D right-hand side, and rho v3 does not change."""
    cells2 = vortex_two_level_cells(2, 1, 3)
    cells3 = extrude_cells(cells2)
    N = 3
    x, _ = lgl_nodes_weights(N)
    U2 = smooth_random_state(cells2, -1.0, L, x, amplitude=0.1)
    K2 = DGSEM(TreeMesh(np.asarray(cells2), -1.0, L), N, flux).rhs(U2)
    index2 = {tuple(c): e for e, c in enumerate(cells2)}
    U3 = np.zeros((len(cells3), 5, N + 1, N + 1, N + 1))
    for e3, (l, ix, iy, iz) in enumerate(cells3):
        u = U2[index2[(l, ix, iy)]]
        U3[e3, [0, 1, 2, 4]] = u[:, None, :, :]
    mesh3 = _mesh(cells3)
    assert len(mesh3.hanging) > 0
    K3 = DGSEM3D(mesh3, N, flux).rhs(U3)
    scale = np.max(np.abs(K2))
    for e3, (l, ix, iy, iz) in enumerate(cells3):
        want = K2[index2[(l, ix, iy)]]
        assert np.max(np.abs(K3[e3, [0, 1, 2, 4]] - want[:, None, :, :])) < 1e-12 * scale
        assert np.max(np.abs(K3[e3, 3])) < 1e-12 * scale


@pytest.mark.parametrize("N", [2, 3])
def test_consistency_order_against_the_exact_density_wave(N):
    """The RHS of the sampled exact solution converges to its time derivative at order >= N
    (asymptotically: the rate between the two finest meshes; the errors fall throughout)."""
    x, w = lgl_nodes_weights(N)
    vel = (0.3, -0.2, 0.5)
    errs = []
    for level in (1, 2, 3):
        cells = uniform_cells3(level)
        U = nodal_state3(density_wave3, cells, -1.0, L, x, period=L, velocity=vel)
        K = DGSEM3D(_mesh(cells), N, "hll").rhs(U)
        eps = 1e-6
        dU = (nodal_state3(density_wave3, cells, -1.0, L, x, t=eps, period=L, velocity=vel)
              - nodal_state3(density_wave3, cells, -1.0, L, x, t=-eps, period=L, velocity=vel)) / (2 * eps)
        mesh = _mesh(cells)
        errs.append(np.sqrt(np.einsum("e,evkji,k,j,i->", (0.5 * mesh.h) ** 3, (K - dU) ** 2, w, w, w)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[0] > errs[1] > errs[2]
    assert rates[-1] > N - 0.4, (errs, rates)


def _asymmetric_cells():
    return refine_cells3(uniform_cells3(2), lambda l, ix, iy, iz: 1 <= ix < 2 and 0 <= iy < 3 and 2 <= iz < 4)


def test_axis_permutation_symmetry():
    """Relabelling the axes (x, y, z) -> (z, x, y) maps the RHS onto the relabelled RHS."""
    cells = _asymmetric_cells()
    N = 3
    x, _ = lgl_nodes_weights(N)
    U = smooth_random_state3(cells, -1.0, L, x, amplitude=0.1)
    K = DGSEM3D(_mesh(cells), N, "hllc").rhs(U)
    # new coordinates (x', y', z') = (y, z, x): cell (l, ix, iy, iz) -> (l, iy, iz, ix)
    cells_p = [(l, iy, iz, ix) for (l, ix, iy, iz) in cells]
    perm_vars = [0, 2, 3, 1, 4]               # (m1', m2', m3') = (m2, m3, m1)

    def relabel(A):
        # A'[e, v', k', j', i'] with i' = j, j' = k, k' = i
        return np.transpose(A, (0, 1, 4, 2, 3))[:, perm_vars]

    Kp = DGSEM3D(_mesh(cells_p), N, "hllc").rhs(relabel(U))
    assert np.max(np.abs(Kp - relabel(K))) < 1e-12 * np.max(np.abs(K))


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_mirror_symmetry(axis):
    """Reflecting the mesh and the state across a coordinate plane reflects the RHS."""
    cells = _asymmetric_cells()
    N = 2
    x, _ = lgl_nodes_weights(N)
    U = smooth_random_state3(cells, -1.0, L, x, amplitude=0.1)
    K = DGSEM3D(_mesh(cells), N, "hll").rhs(U)
    cells_m = []
    for c in cells:
        c = list(c)
        c[1 + axis] = (1 << c[0]) - 1 - c[1 + axis]
        cells_m.append(tuple(c))
    spatial = 4 - axis                           # array axis of the mirrored coordinate

    def mirror(A):
        B = np.flip(A, axis=spatial).copy()
        B[:, 1 + axis] *= -1.0
        return B

    Km = DGSEM3D(_mesh(cells_m), N, "hll").rhs(mirror(U))
    assert np.max(np.abs(Km - mirror(K))) < 1e-12 * np.max(np.abs(K))


def test_face_projection_is_exact_on_polynomials_and_separable():
    N = 3
    x, _ = lgl_nodes_weights(N)
    rng = np.random.default_rng(5)
    C = rng.normal(size=(N + 1, N + 1))           # coefficients of a Q_N polynomial in monomials
    def poly(s1, s2):
        return sum(C[b, a] * s1 ** a * s2 ** b for a in range(N + 1) for b in range(N + 1))
    quads = {}
    for q1 in (0, 1):
        for q2 in (0, 1):
            s1 = 0.5 * (x + (2 * q1 - 1))
            s2 = 0.5 * (x + (2 * q2 - 1))
            quads[(q1, q2)] = poly(s1[None, :], s2[:, None])
    got = face_l2_projection(x, quads)
    assert np.max(np.abs(got - poly(x[None, :], x[:, None]))) < 1e-12 * np.max(np.abs(got))
    # piecewise data: the projection equals the 1D two-halves projection along t1, then along t2
    pieces = {k: rng.normal(size=(2, N + 1, N + 1)) for k in quads}
    got = face_l2_projection(x, pieces)
    rows = {q2: l2_project_two_halves(x, pieces[(0, q2)], pieces[(1, q2)]) for q2 in (0, 1)}   # along t1
    want = np.swapaxes(l2_project_two_halves(x, np.swapaxes(rows[0], -1, -2), np.swapaxes(rows[1], -1, -2)),
                       -1, -2)
    assert np.max(np.abs(got - want)) < 1e-12


@pytest.mark.parametrize("flux", [euler3d.hll_flux, euler3d.hllc_flux, euler3d.hlle_flux, euler3d.ec_flux])
def test_fluxes_consistent_and_reduce_to_2d(flux):
    rng = np.random.default_rng(11)
    n = 64
    prim = [rng.uniform(0.5, 2.0, n), rng.normal(0, 0.5, n), rng.normal(0, 0.5, n), np.zeros(n),
            rng.uniform(0.5, 2.0, n)]
    u = prim_to_cons3(*prim)
    primR = [rng.uniform(0.5, 2.0, n), rng.normal(0, 0.5, n), rng.normal(0, 0.5, n), np.zeros(n),
             rng.uniform(0.5, 2.0, n)]
    uR = prim_to_cons3(*primR)
    flux2 = {euler3d.hll_flux: euler.hll_flux, euler3d.hllc_flux: euler.hllc_flux,
             euler3d.hlle_flux: euler.hlle_flux, euler3d.ec_flux: euler.ec_flux}[flux]
    for d in range(3):
        assert np.allclose(flux(u, u, d), euler3d.physical_flux(u, d), rtol=1e-13, atol=1e-13)
    for d in range(2):
        f3 = flux(u, uR, d)
        f2 = flux2(u[[0, 1, 2, 4]], uR[[0, 1, 2, 4]], d)
        assert np.allclose(f3[[0, 1, 2, 4]], f2, rtol=1e-13, atol=1e-14)
        assert np.max(np.abs(f3[3])) < 1e-14


@pytest.mark.parametrize("flux", [euler3d.hll_flux, euler3d.hllc_flux, euler3d.hlle_flux, euler3d.ec_flux])
def test_fluxes_rotation_invariant(flux):
    """The flux along z of a state equals the flux along x of the state with axes relabelled."""
    rng = np.random.default_rng(12)
    n = 64
    uL = prim_to_cons3(rng.uniform(0.5, 2, n), *rng.normal(0, 0.5, (3, n)), rng.uniform(0.5, 2, n))
    uR = prim_to_cons3(rng.uniform(0.5, 2, n), *rng.normal(0, 0.5, (3, n)), rng.uniform(0.5, 2, n))
    perm = [0, 3, 1, 2, 4]                 # z becomes x: (m1', m2', m3') = (m3, m1, m2)
    fz = flux(uL, uR, 2)
    fx = flux(uL[perm], uR[perm], 0)
    assert np.allclose(fz[perm], fx, rtol=1e-13, atol=1e-14)


def test_ec_flux_entropy_conservative_3d():
    rng = np.random.default_rng(13)
    n = 256
    uL = prim_to_cons3(rng.uniform(0.5, 2, n), *rng.normal(0, 0.5, (3, n)), rng.uniform(0.5, 2, n))
    uR = prim_to_cons3(rng.uniform(0.5, 2, n), *rng.normal(0, 0.5, (3, n)), rng.uniform(0.5, 2, n))
    for d in range(3):
        f = euler3d.ec_flux(uL, uR, d)
        lhs = np.sum((euler3d.entropy_variables(uR) - euler3d.entropy_variables(uL)) * f, axis=0)
        rhs = euler3d.entropy_flux_potential(uR, d) - euler3d.entropy_flux_potential(uL, d)
        assert np.max(np.abs(lhs - rhs)) < 1e-12


def test_hllc_resolves_a_stationary_contact():
    n = 8
    rng = np.random.default_rng(14)
    p = 1.3
    uL = prim_to_cons3(rng.uniform(0.5, 2, n), np.zeros(n), rng.normal(0, 1, n), rng.normal(0, 1, n), p * np.ones(n))
    uR = prim_to_cons3(rng.uniform(0.5, 2, n), np.zeros(n), rng.normal(0, 1, n), rng.normal(0, 1, n), p * np.ones(n))
    f = euler3d.hllc_flux(uL, uR, 0)
    want = np.zeros_like(f)
    want[1] = p
    assert np.max(np.abs(f - want)) < 1e-13


def test_dt_rule_closed_form():
    cells = uniform_cells3(1)
    x, _ = lgl_nodes_weights(2)
    U = np.empty((8, 5, 3, 3, 3))
    U[:] = prim_to_cons3(1.0, 0.3, -0.4, 0.5, 1.0)[None, :, None, None, None]
    c = math.sqrt(1.4)
    h = np.full(8, 1.0)
    assert abs(max_wave_speed_dt3(U, h, 2, 0.5) - 0.5 * 1.0 / (3 * (1.2 + 3 * c))) < 1e-15


def test_single_level_perk3_step_is_the_standalone_method():
    """With one level the P-ERK3 family's finest member integrates every element: the dense
    partitioned step equals the standalone member applied to the whole 3D system."""
    cells = uniform_cells3(1)
    x, _ = lgl_nodes_weights(2)
    U = smooth_random_state3(cells, -1.0, L, x, amplitude=0.1)
    op = DGSEM3D(_mesh(cells), 2, "hlle")
    fam = perk3_family([3, 4, 6])
    meth = element_methods(np.asarray(cells)[:, 0], fam.R)
    assert np.all(meth == fam.R - 1)
    got = prkm_step(op.rhs, U, 0.01, fam, meth)
    A = fam.A[fam.R - 1]
    K = []
    for i in range(fam.S):
        Y = U + 0.01 * sum(A[i, j] * K[j] for j in range(i)) if i else U.copy()
        K.append(op.rhs(Y))
    want = U + 0.01 * sum(fam.b[i] * K[i] for i in range(fam.S))
    assert np.max(np.abs(got - want)) < 1e-14 * np.max(np.abs(U))
