"""Pins of the oracle's LGL operators against closed forms and textbook identities."""
import math

import numpy as np
import pytest

from oracle.lgl import (derivative_matrix, l2_project_two_halves, lagrange_eval, lgl_nodes_weights,
                        mass_matrix_exact)


def test_lgl_n3_closed_form():
    # N = 3: nodes -1, -1/sqrt(5), 1/sqrt(5), 1 and weights 1/6, 5/6, 5/6, 1/6
    x, w = lgl_nodes_weights(3)
    s = 1.0 / math.sqrt(5.0)
    np.testing.assert_allclose(x, [-1.0, -s, s, 1.0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], rtol=0, atol=1e-15)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 6])
def test_quadrature_exactness(N):
    # N+1 LGL points integrate polynomials up to degree 2N-1 exactly
    x, w = lgl_nodes_weights(N)
    for k in range(2 * N):
        exact = (1.0 - (-1.0) ** (k + 1)) / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14


@pytest.mark.parametrize("N", [2, 3, 5])
def test_derivative_exact_on_polynomials(N):
    x, _ = lgl_nodes_weights(N)
    D = derivative_matrix(x)
    for k in range(N + 1):
        d = k * x ** (k - 1) if k > 0 else 0 * x
        np.testing.assert_allclose(D @ x ** k, d, atol=1e-13)


@pytest.mark.parametrize("N", [2, 3, 5])
def test_summation_by_parts(N):
    # W D + (W D)^T = diag(-1, 0, ..., 0, 1)
    x, w = lgl_nodes_weights(N)
    Q = np.diag(w) @ derivative_matrix(x)
    B = np.zeros((N + 1, N + 1))
    B[0, 0], B[N, N] = -1.0, 1.0
    np.testing.assert_allclose(Q + Q.T, B, atol=1e-14)


def test_mass_matrix_against_legendre_orthogonality():
    # exact mass matrix of the Lagrange basis reproduces int x^a x^b for a + b <= 2N
    N = 3
    x, _ = lgl_nodes_weights(N)
    M = mass_matrix_exact(x)
    for a in range(N + 1):
        for b in range(N + 1):
            exact = (1.0 - (-1.0) ** (a + b + 1)) / (a + b + 1)
            assert abs((x ** a) @ M @ (x ** b) - exact) < 1e-14


def test_l2_projection_reproduces_polynomials_and_conserves():
    N = 3
    x, w = lgl_nodes_weights(N)
    rng = np.random.default_rng(0)
    coef = rng.normal(size=N + 1)
    poly = lambda t: np.polyval(coef, t)
    # a global degree-N polynomial split into its two halves projects back onto itself
    lower = poly(0.5 * (x - 1.0))
    upper = poly(0.5 * (x + 1.0))
    np.testing.assert_allclose(l2_project_two_halves(x, lower, upper), poly(x), atol=1e-13)
    # a discontinuous piecewise polynomial keeps its integral (test function 1)
    lower = rng.normal(size=N + 1)
    upper = rng.normal(size=N + 1)
    phi = l2_project_two_halves(x, lower, upper)
    assert abs(np.dot(w, phi) - 0.5 * (np.dot(w, lower) + np.dot(w, upper))) < 1e-14
    # and is orthogonal to its own residual: int (phi - f) x^k = 0 for k <= N
    xg, wg = np.polynomial.legendre.leggauss(8)
    for k in range(N + 1):
        r = 0.0
        for f, shift in ((lower, -0.5), (upper, 0.5)):
            xp = 0.5 * xg + shift
            r += np.sum(0.5 * wg * (lagrange_eval(x, phi, xp) - lagrange_eval(x, f, xg)) * xp ** k)
        assert abs(r) < 1e-14
