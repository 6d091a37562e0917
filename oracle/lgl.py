"""Legendre-Gauss-Lobatto (LGL) collocation on [-1, 1] (oracle; test infrastructure only).

The DGSEM the paper uses (Sec. 6.1, with flux differencing, and the TreeMesh
mortars of Sec. 6.2) collocates the solution at the N+1 LGL nodes: the end
points plus the roots of P_N'.  Everything here is the textbook definition:
Lagrange polynomials as products, their derivatives as the derivative of the
product, and integrals by Gauss-Legendre quadrature exact for the integrand's
degree.
"""

from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg


def lgl_nodes_weights(N: int):
    """Nodes x_0 < ... < x_N (end points and roots of P_N') and weights
    w_i = 2 / (N (N+1) P_N(x_i)^2)."""
    PN = npleg.Legendre.basis(N)
    dPN = PN.deriv()
    inner = np.sort(np.real(dPN.roots())) if N > 1 else np.array([])
    d2PN = dPN.deriv()
    for _ in range(3):  # polish the interior roots with Newton steps on P_N'
        inner = inner - dPN(inner) / d2PN(inner)
    x = np.concatenate([[-1.0], inner, [1.0]])
    w = 2.0 / (N * (N + 1) * PN(x) ** 2)
    return x, w


def lagrange_basis(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """L[k, j] = l_j(x_k) with l_j(x) = prod_{m != j} (x - x_m) / (x_j - x_m)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    L = np.ones((len(x), n))
    for j in range(n):
        for m in range(n):
            if m != j:
                L[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
    return L


def lagrange_eval(nodes: np.ndarray, values: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Interpolant through (nodes, values[..., j]) evaluated at x: returns [..., len(x)]."""
    return np.asarray(values) @ lagrange_basis(nodes, x).T


def derivative_matrix(nodes: np.ndarray) -> np.ndarray:
    """D[i, j] = l_j'(x_i), from differentiating the product form of l_j:
    l_j'(x_i) = prod_{m != i, j}(x_i - x_m) / prod_{m != j}(x_j - x_m) for i != j
    and l_i'(x_i) = sum_{m != i} 1 / (x_i - x_m)."""
    x = np.asarray(nodes, dtype=np.float64)
    n = len(x)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i == j:
                D[i, i] = sum(1.0 / (x[i] - x[m]) for m in range(n) if m != i)
            else:
                num = 1.0
                den = 1.0
                for m in range(n):
                    if m != j:
                        den *= x[j] - x[m]
                    if m != i and m != j:
                        num *= x[i] - x[m]
                D[i, j] = num / den
    return D


def mass_matrix_exact(nodes: np.ndarray) -> np.ndarray:
    """M[j, k] = integral_{-1}^{1} l_j l_k dx, by Gauss-Legendre quadrature with
    len(nodes) points (exact for the degree-2N integrand)."""
    xg, wg = npleg.leggauss(len(nodes))
    L = lagrange_basis(nodes, xg)
    return L.T @ (wg[:, None] * L)


def l2_project_two_halves(nodes: np.ndarray, f_lower: np.ndarray, f_upper: np.ndarray) -> np.ndarray:
    """L2 projection onto degree-N polynomials on [-1, 1] of the piecewise
    polynomial equal to the interpolant of ``f_lower`` on [-1, 0] and of
    ``f_upper`` on [0, 1] (each given at the nodes mapped onto its half).

    Solves M phi = b with b_k = int_{-1}^{0} f_lower l_k + int_{0}^{1} f_upper l_k,
    both integrals by Gauss quadrature on the half interval.  The last axis of
    f_lower / f_upper is the node index.
    """
    n = len(nodes)
    xg, wg = npleg.leggauss(n + 1)
    M = mass_matrix_exact(nodes)
    b = 0.0
    for f, shift in ((f_lower, -0.5), (f_upper, 0.5)):
        # physical points on the half interval and their reference position s on [-1, 1]
        xphys = 0.5 * xg + shift
        f_at = lagrange_eval(nodes, f, xg)                  # f as function of s at Gauss points
        lk = lagrange_basis(nodes, xphys)                   # l_k at the physical points
        b = b + (f_at * (0.5 * wg)) @ lk                    # dx = ds / 2
    b = np.asarray(b)
    phi = np.linalg.solve(M, b.reshape(-1, n).T).T
    return phi.reshape(b.shape)
