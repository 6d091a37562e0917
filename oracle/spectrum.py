"""Spectrum-optimised stability polynomials (oracle; test infrastructure only).

Sec. 4 of the paper: a member with E stage evaluations and linear order p has
the stability polynomial

    P(z) = sum_{i=0}^{p} z^i / i!  +  sum_{i=p+1}^{E} alpha_i z^i,

and alpha is chosen to maximise dt subject to |P(dt lambda)| <= 1 for every
lambda of a set sigma of eigenvalues of the semidiscretisation's Jacobian
(Eq. OptimizationProblem).  For a fixed dt the constraints are convex in alpha
(Ketcheson & Ahmadia 2012); the largest dt is found by bisection over such
feasibility problems.  Each feasibility problem is solved here as a sequence
of linear programs: |w| <= 1 is the intersection of the half planes
Re(w e^{-i theta}) <= 1 over all theta; the LP starts from a few theta per
eigenvalue and adds, for every eigenvalue whose current |P| exceeds 1, the
half plane at theta = arg P (a cutting-plane method), until no constraint is
violated by more than a tolerance or the LP becomes infeasible.

The spectrum sigma: the eigenvalues of the dense Jacobian of a small
semidiscretisation (Sec. 4.1, step 1), reduced to the points of their convex
hull in the closed second quadrant (the spectrum is symmetric about the real
axis) with extra points on long hull edges so that no two neighbours are
farther apart than the mean hull-edge length (step 2).
"""

from __future__ import annotations

import math

import numpy as np
from scipy.optimize import linprog
from scipy.spatial import ConvexHull


def fixed_part(z: np.ndarray, p: int) -> np.ndarray:
    """sum_{i<=p} z^i / i! at the points z."""
    out = np.zeros_like(z, dtype=complex)
    for i in range(p + 1):
        out = out + z ** i / math.factorial(i)
    return out


def polynomial_values(z: np.ndarray, p: int, alpha: np.ndarray) -> np.ndarray:
    """P(z) with free coefficients alpha[k] of z^{p+1+k}."""
    out = fixed_part(z, p)
    for k, a in enumerate(alpha):
        out = out + a * z ** (p + 1 + k)
    return out


def feasible_coefficients(z: np.ndarray, E: int, p: int, tol: float = 1e-10, max_rounds: int = 400):
    """alpha with max |P(z_k)| <= 1 + tol, or None if none exists.

    Cutting planes on the min-max problem: minimise s subject to
    Re(e^{-i theta} P(z_k)) <= s over the half planes collected so far.  This is
    a relaxation of min_alpha max_k |P(z_k)|, so an optimum s > 1 proves that no
    alpha is feasible; otherwise the half plane at theta = arg P(z_k) is added for
    every eigenvalue with |P(z_k)| > 1 + tol and the LP is solved again.  The
    unknowns are scaled, beta_k = alpha_k R^{p+1+k} with R = max |z|, so that the
    LP matrix entries are bounded by one."""
    z = np.asarray(z, dtype=complex)
    n = E - p
    T = fixed_part(z, p)
    if n <= 0:
        return np.zeros(0) if np.all(np.abs(T) <= 1.0 + tol) else None
    R = max(np.max(np.abs(z)), 1e-300)
    powers = np.stack([(z / R) ** (p + 1 + k) for k in range(n)], axis=1)   # [K, n]
    rows_k = np.concatenate([np.arange(len(z))] * 8)
    rows_t = np.concatenate([np.full(len(z), 2.0 * math.pi * j / 8.0) for j in range(8)])
    c = np.zeros(n + 1)
    c[-1] = 1.0
    for _ in range(max_rounds):
        rot = np.exp(-1j * rows_t)
        A = np.concatenate([np.real(rot[:, None] * powers[rows_k]), -np.ones((len(rows_k), 1))], axis=1)
        b = -np.real(rot * T[rows_k])
        res = linprog(c, A_ub=A, b_ub=b, bounds=[(None, None)] * (n + 1), method="highs")
        if res.status != 0:
            return None
        if res.x[-1] > 1.0 + tol:
            return None
        beta = res.x[:n]
        w = T + powers @ beta
        viol = np.abs(w) > 1.0 + tol
        if not np.any(viol):
            return beta / R ** (p + 1 + np.arange(n))
        idx = np.nonzero(viol)[0]
        rows_k = np.concatenate([rows_k, idx])
        rows_t = np.concatenate([rows_t, np.angle(w[idx])])
    return None


def optimal_polynomial(sigma: np.ndarray, E: int, p: int, rel_tol: float = 1e-7):
    """(dt_max, alpha) of Eq. OptimizationProblem by bisection on dt."""
    sigma = np.asarray(sigma, dtype=complex)
    sigma = sigma[np.abs(sigma) > 0]
    lam = np.max(np.abs(sigma))
    lo, hi = 0.0, 4.0 * E * E / lam
    best = None
    # grow lo from a small feasible value
    t = 1e-3 / lam
    while t < hi:
        a = feasible_coefficients(t * sigma, E, p)
        if a is None:
            hi = t
            break
        lo, best = t, a
        t *= 2.0
    if best is None:
        return 0.0, None
    while hi - lo > rel_tol * lo:
        mid = 0.5 * (lo + hi)
        a = feasible_coefficients(mid * sigma, E, p)
        if a is None:
            hi = mid
        else:
            lo, best = mid, a
    return lo, best


def hull_points(eigs: np.ndarray, eps: float = 1e-12) -> np.ndarray:
    """Convex-hull points of the eigenvalues in the closed second quadrant, refined so that
    consecutive points are no farther apart than the mean hull-edge length (Sec. 4.1, step 2)."""
    e = np.asarray(eigs, dtype=complex)
    q = e[(e.real <= eps) & (e.imag >= -eps)]
    pts = np.stack([q.real, np.maximum(q.imag, 0.0)], axis=1)
    pts = np.concatenate([pts, [[0.0, 0.0]]])
    hull = ConvexHull(pts)
    v = pts[hull.vertices]                       # counter-clockwise
    edges = [(v[k], v[(k + 1) % len(v)]) for k in range(len(v))]
    lengths = [np.linalg.norm(b - a) for a, b in edges]
    delta = float(np.mean(lengths))
    out = []
    for (a, b), L in zip(edges, lengths):
        m = max(1, int(math.ceil(L / delta)))
        for s in range(m):
            out.append(a + (b - a) * s / m)
    out = np.array(out)
    return out[:, 0] + 1j * out[:, 1]


def dense_jacobian(rhs, U: np.ndarray) -> np.ndarray:
    """The Jacobian of the flattened rhs at U by automatic differentiation (torch, float64)."""
    import torch

    x = torch.tensor(np.asarray(U, dtype=np.float64).reshape(-1), requires_grad=False)
    J = torch.autograd.functional.jacobian(lambda v: rhs(v.reshape(U.shape)).reshape(-1), x)
    return J.numpy()
