"""Pins of the oracle's Euler fluxes: consistency, symmetry, entropy conservation,
upwinding and exact resolution of isolated discontinuities."""
import numpy as np
import pytest

from oracle import euler

G = euler.GAMMA


def cons(rho, v1, v2, p):
    return np.array([rho, rho * v1, rho * v2, p / (G - 1) + 0.5 * rho * (v1 * v1 + v2 * v2)], dtype=float)


def random_states(n, seed):
    rng = np.random.default_rng(seed)
    return cons(rng.uniform(0.3, 2, n), rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(0.3, 2, n))


def test_log_mean_closed_forms():
    # ln-mean of (a, a e) is a (e - 1); symmetric; equal arguments return the argument
    a = np.array([0.5, 1.0, 3.0])
    np.testing.assert_allclose(euler.log_mean(a, a * np.e), a * (np.e - 1), rtol=1e-15)
    np.testing.assert_allclose(euler.log_mean(a, 2 * a), euler.log_mean(2 * a, a), rtol=1e-15)
    np.testing.assert_array_equal(euler.log_mean(a, a), a)
    # near-equal arguments: the mean of (1, 1 + d) is 1 + d/2 - d^2/12 + O(d^3)
    b = 1.0 + 1e-7
    d = b - 1.0                      # exact in floating point
    assert abs(euler.log_mean(1.0, b) - (1 + d / 2 - d * d / 12)) < 4e-16


@pytest.mark.parametrize("d", [0, 1])
def test_two_point_flux_consistent_symmetric(d):
    uL = random_states(50, 1)
    uR = random_states(50, 2)
    np.testing.assert_allclose(euler.ec_flux(uL, uL, d), euler.physical_flux(uL, d), rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(euler.ec_flux(uL, uR, d), euler.ec_flux(uR, uL, d), rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("d", [0, 1])
def test_two_point_flux_entropy_conservative(d):
    # Tadmor's condition (w_R - w_L) . f#(u_L, u_R) = psi_R - psi_L
    uL = random_states(200, 3)
    uR = random_states(200, 4)
    lhs = np.sum((euler.entropy_variables(uR) - euler.entropy_variables(uL)) * euler.ec_flux(uL, uR, d), axis=0)
    rhs = euler.entropy_flux_potential(uR, d) - euler.entropy_flux_potential(uL, d)
    np.testing.assert_allclose(lhs, rhs, atol=1e-13)


@pytest.mark.parametrize("flux", [euler.hll_flux, euler.hllc_flux])
@pytest.mark.parametrize("d", [0, 1])
def test_surface_flux_consistency_and_upwinding(flux, d):
    u = random_states(20, 5)
    np.testing.assert_allclose(flux(u, u, d), euler.physical_flux(u, d), rtol=1e-14, atol=1e-14)
    # supersonic to the right: the flux is the left physical flux
    uL = cons(1.0, 5.0, 5.0, 1.0)
    uR = cons(0.5, 4.0, 4.0, 0.8)
    np.testing.assert_allclose(flux(uL, uR, d), euler.physical_flux(uL, d), rtol=1e-15)
    # supersonic to the left: the right physical flux
    uL = cons(1.0, -5.0, -5.0, 1.0)
    uR = cons(0.5, -4.0, -4.0, 0.8)
    np.testing.assert_allclose(flux(uL, uR, d), euler.physical_flux(uR, d), rtol=1e-15)


@pytest.mark.parametrize("d", [0, 1])
def test_hllc_resolves_contact(d):
    # isolated contact (density jump, equal normal velocity and pressure): HLLC gives the exact flux
    v = 0.3
    vel = (v, 0.7) if d == 0 else (0.7, v)
    uL = cons(1.0, *vel, 1.0)
    uR = cons(0.25, *vel, 1.0)
    f = euler.hllc_flux(uL, uR, d)
    np.testing.assert_allclose(f, euler.physical_flux(uL, d), rtol=1e-14)
    # HLL smears it: its mass flux lies strictly between the two sides' exact ones
    fh = euler.hll_flux(uL, uR, d)
    assert abs(fh[0] - f[0]) > 1e-3


def test_hll_mass_flux_formula():
    # subsonic HLL mass flux from the formula with Davis speeds written out
    uL = cons(1.0, 0.2, 0.0, 1.0)
    uR = cons(0.5, -0.1, 0.0, 0.6)
    cL, cR = np.sqrt(G * 1.0 / 1.0), np.sqrt(G * 0.6 / 0.5)
    SL, SR = min(0.2 - cL, -0.1 - cR), max(0.2 + cL, -0.1 + cR)
    f_expect = (SR * 0.2 - SL * (-0.05) + SL * SR * (0.5 - 1.0)) / (SR - SL)
    assert abs(euler.hll_flux(uL, uR, 0)[0] - f_expect) < 1e-15
