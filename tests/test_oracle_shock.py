"""Pins of the subcell shock capturing and the HLLE flux of the oracle (oracle/shock.py,
oracle/euler.py) against properties the mathematics fixes."""

import math

import numpy as np
import pytest

from oracle import euler
from oracle.lgl import lgl_nodes_weights
from oracle.shock import ShockCapturingDGSEM, blending_factor, finite_volume_term, legendre_vandermonde
from oracle.dgsem import DGSEM
from oracle.treemesh import TreeMesh
from perk_inputs import kh_band_cells, nodal_state, uniform_cells, vortex_two_level_cells
from perk_inputs import kelvin_helmholtz

X, W = lgl_nodes_weights(3)


def random_states(n, seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.3, 2.0, n)
    v1, v2 = rng.uniform(-1.0, 1.0, (2, n))
    p = rng.uniform(0.3, 3.0, n)
    return np.stack([rho, rho * v1, rho * v2, p / 0.4 + 0.5 * rho * (v1 * v1 + v2 * v2)])


def test_hlle_consistency_and_speeds():
    u = random_states(50, 1)
    for d in (0, 1):
        np.testing.assert_allclose(euler.hlle_flux(u, u, d), euler.physical_flux(u, d), rtol=1e-14, atol=1e-14)
        SL, SR = euler.einfeldt_speeds(u, u, d)
        rho, v1, v2, p = euler.primitives(u)
        c = np.sqrt(1.4 * p / rho)
        vn = v1 if d == 0 else v2
        np.testing.assert_allclose(SL, vn - c, rtol=1e-13)
        np.testing.assert_allclose(SR, vn + c, rtol=1e-13)


def test_hlle_is_entropy_stable():
    # (w_R - w_L) . (f* - f_EC) <= 0 for every pair: the flux dissipates entropy relative to the
    # entropy-conservative two-point flux (Tadmor)
    uL, uR = random_states(400, 2), random_states(400, 3)
    for d in (0, 1):
        dw = euler.entropy_variables(uR) - euler.entropy_variables(uL)
        prod = np.sum(dw * (euler.hlle_flux(uL, uR, d) - euler.ec_flux(uL, uR, d)), axis=0)
        assert np.all(prod <= 1e-12)


def state_with_pressure(eps_line):
    """rho = 1, v = 0, p = eps along x (constant in y): U [1, 4, 4, 4]."""
    U = np.zeros((1, 4, 4, 4))
    U[0, 0] = 1.0
    U[0, 3] = np.tile(eps_line, (4, 1)) / 0.4
    return U


def test_blending_factor_closed_forms():
    V = legendre_vandermonde(X)
    T = 0.5 * 10.0 ** (-1.8 * 4 ** 0.25)
    s = math.log((1.0 - 1e-4) / 1e-4)
    for frac, want in ((T, 0.5), (0.5 * T, 1.0 / (1.0 + math.exp(0.5 * s)))):
        # epsilon = c0 L_0 + c3 L_3 with c3^2 / (c0^2 + c3^2) = frac: the share of the top mode
        c0 = 1.0
        c3 = math.sqrt(frac / (1.0 - frac))
        eps = V @ np.array([c0, 0.0, 0.0, c3])
        got = blending_factor(state_with_pressure(eps), X, alpha_max=1.0)[0]
        assert abs(got - want) < 1e-10
    # linear data has no energy above mode 1: alpha = 0; the cap applies to a pure top mode
    assert blending_factor(state_with_pressure(1.0 + 0.3 * X), X)[0] == 0.0
    assert blending_factor(state_with_pressure(V @ np.array([1.0, 0.0, 0.0, 5.0])), X)[0] == 0.5
    # the indicator is invariant under scaling of epsilon and under exchanging x and y
    eps = 1.0 + 0.2 * np.sin(3.0 * X)
    a1 = blending_factor(state_with_pressure(eps), X, alpha_max=1.0)[0]
    a2 = blending_factor(state_with_pressure(7.0 * eps), X, alpha_max=1.0)[0]
    Ut = state_with_pressure(eps)
    Ut[0, 3] = Ut[0, 3].T
    a3 = blending_factor(Ut, X, alpha_max=1.0)[0]
    assert abs(a1 - a2) < 1e-12 and abs(a1 - a3) < 1e-12


def test_finite_volume_term_telescopes_and_vanishes_on_constants():
    U = random_states(3 * 16, 5).reshape(4, 3, 4, 4)                                  # [4, e, j, i]
    # for data constant in y only the x part remains; along each grid line
    # sum_i w_i T_i = f(u_N) - f(u_0) (the subcell fluxes telescope)
    Uy = np.repeat(U[:, :, :1, :], 4, axis=2)
    T = finite_volume_term(Uy, W, euler.hlle_flux)
    lhs = np.einsum("i,veji->vej", W, T)
    rhs = euler.physical_flux(Uy[..., 3], 0) - euler.physical_flux(Uy[..., 0], 0)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)
    const = np.ones_like(U) * U[:, :1, :1, :1]
    assert np.max(np.abs(finite_volume_term(const, W, euler.hlle_flux))) < 1e-12


def test_blended_rhs_free_stream_conservation_entropy():
    # free stream at hanging faces
    cells = vortex_two_level_cells(3, 2, 6)
    m = TreeMesh(cells, 0.0, 1.0)
    U = np.zeros((len(cells), 4, 4, 4))
    U[:, 0], U[:, 1], U[:, 2], U[:, 3] = 1.2, 0.3, -0.24, 3.0
    assert np.max(np.abs(ShockCapturingDGSEM(m, 3, "hlle").rhs(U))) < 1e-12
    # a discontinuous state: some alpha > 0; conservation on the non-conforming mesh
    U = np.moveaxis(random_states(len(cells) * 16, 7).reshape(4, len(cells), 4, 4), 0, 1).copy()
    sc = ShockCapturingDGSEM(m, 3, "hlle")
    assert np.max(blending_factor(U, X)) == 0.5
    K = sc.rhs(U)
    tot = sc.integrate(K)
    assert np.max(np.abs(tot)) < 1e-12 * np.max(np.abs(sc.integrate(np.abs(K))))
    # entropy: EC volume + HLLE surfaces + HLLE subcells dissipate (conforming periodic mesh)
    cc = uniform_cells(2)
    mc = TreeMesh(cc, 0.0, 1.0)
    Uc = np.moveaxis(random_states(len(cc) * 16, 8).reshape(4, len(cc), 4, 4), 0, 1).copy()
    Kc = ShockCapturingDGSEM(mc, 3, "hlle").rhs(Uc)
    wv = np.moveaxis(euler.entropy_variables(np.moveaxis(Uc, 1, 0)), 0, 1)
    dS = np.einsum("e,evji,ji->", (0.5 * mc.h) ** 2, wv * Kc, np.outer(W, W))
    assert dS < 0.0


def test_blend_is_the_plain_dgsem_where_alpha_is_zero():
    cells = kh_band_cells(3, 4, 0.1)
    m = TreeMesh(cells, -1.0, 2.0)
    U = nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X)
    alpha = blending_factor(U, X)
    K1 = ShockCapturingDGSEM(m, 3, "hlle").rhs(U)
    K0 = DGSEM(m, 3, "hlle").rhs(U)
    flat = alpha == 0.0
    assert np.any(flat)
    assert np.array_equal(K1[flat], K0[flat])
