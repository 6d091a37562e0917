"""Stability polynomials optimised for the spectrum of the discretisation (Sec. 4).

The library's Jacobian apply (``perk_rhs_jvp``, the K-JVP kernels) is the only
operator used:

* ``jacobian_dense``: J(U) column by column, for a small mesh whose full
  eigendecomposition is cheap (the reduced system of Sec. 4.1, step 1);
* ``ritz_values``: an Arnoldi iteration on the GPU (modified Gram-Schmidt with
  one re-orthogonalisation) whose Ritz values approximate the outer
  eigenvalues of J(U) on the full mesh.  The paper runs shifted Arnoldi
  iterations on a stored sparse Jacobian (Sec. 4.1, steps 3-4); here the
  Jacobian is never formed, so the outer Ritz values of the unshifted
  iteration stand in for them, and the reduced spectrum scaled by the ratio of
  the finest cell sizes supplies the rest of the boundary;
* ``boundary``: the convex hull of eigenvalues in the closed second quadrant,
  refined so that neighbours are no farther apart than the mean hull edge
  (Sec. 4.1, step 2);
* ``optimize``: Eq. OptimizationProblem.  For a fixed dt the constraints
  |P(dt lambda)| <= 1 are convex in the free coefficients; dt is found by
  bisection, and each feasibility question is answered by minimising
  s subject to |P(dt lambda_k)|^2 <= s (smooth convex constraints, SLSQP);
* ``perk2_family_from_spectrum``: members of a second-order family built from
  the optimised polynomials by ``perk2_member`` (Sec. 4.3.1).
"""

from __future__ import annotations

import math
from typing import Sequence

import numpy as np


def jacobian_dense(solver, U, stage: int = -1) -> np.ndarray:
    """J(U) of the (partitioned) RHS as a dense [n, n] matrix, n = n_elem * 64, one JVP per column."""
    torch = solver.torch
    n = U.numel()
    J = np.empty((n, n))
    V = torch.zeros_like(U)
    Kd = torch.empty_like(U)
    flatV = V.view(-1)
    for j in range(n):
        flatV.zero_()
        flatV[j] = 1.0
        solver.rhs_jvp(U, V, stage=stage, out=Kd)
        J[:, j] = Kd.view(-1).cpu().numpy()
    return J


def ritz_values(solver, U, m: int = 200, seed: int = 20240308) -> np.ndarray:
    """Ritz values of J(U) after m Arnoldi steps from a seeded random start vector."""
    torch = solver.torch
    n = U.numel()
    m = min(m, n)
    g = torch.Generator(device="cpu").manual_seed(seed)
    Q = torch.zeros((m + 1, n), dtype=torch.float64, device=U.device)
    H = np.zeros((m + 1, m))
    q = torch.randn(n, generator=g, dtype=torch.float64).to(U.device)
    Q[0] = q / torch.linalg.vector_norm(q)
    w = torch.empty_like(U)
    k_used = m
    for k in range(m):
        solver.rhs_jvp(U, Q[k].view_as(U), out=w)
        v = w.reshape(-1).clone()
        for _ in range(2):                                # Gram-Schmidt twice
            h = Q[: k + 1] @ v
            v -= Q[: k + 1].T @ h
            H[: k + 1, k] += h.cpu().numpy()
        beta = float(torch.linalg.vector_norm(v))
        H[k + 1, k] = beta
        if beta < 1e-12 * max(1.0, np.abs(H[: k + 1, k]).max()):
            k_used = k + 1
            break
        Q[k + 1] = v / beta
    return np.linalg.eigvals(H[:k_used, :k_used])


def boundary(eigs: np.ndarray, tol: float = 1e-12) -> np.ndarray:
    """Refined convex-hull points of the eigenvalues with Re <= 0 in the upper half plane."""
    from scipy.spatial import ConvexHull

    e = np.asarray(eigs, dtype=complex)
    e = e[e.real <= tol]
    pts = np.unique(np.round(np.stack([e.real, np.abs(e.imag)], axis=1), 14), axis=0)
    pts = np.vstack([pts, [0.0, 0.0]])
    hv = pts[ConvexHull(pts).vertices]
    nxt = np.roll(hv, -1, axis=0)
    lengths = np.linalg.norm(nxt - hv, axis=1)
    mean = lengths.mean()
    out = []
    for a, b, L in zip(hv, nxt, lengths):
        pieces = max(1, int(math.ceil(L / mean)))
        t = np.arange(pieces)[:, None] / pieces
        out.append(a + t * (b - a))
    pts = np.vstack(out)
    return pts[:, 0] + 1j * pts[:, 1]


def _taylor(z: np.ndarray, p: int) -> np.ndarray:
    acc = np.ones_like(z)
    term = np.ones_like(z)
    for i in range(1, p + 1):
        term = term * z / i
        acc = acc + term
    return acc


def _min_max_modulus(z: np.ndarray, E: int, p: int):
    """min over the free coefficients of max_k |P(z_k)|^2 and the minimiser (scaled basis)."""
    from scipy.optimize import minimize

    n = E - p
    T = _taylor(z, p)
    R = np.abs(z).max()
    M = np.stack([(z / R) ** (p + 1 + k) for k in range(n)], axis=1)        # [K, n]
    Mr, Mi = M.real, M.imag

    def cons(x):
        w = T + M @ x[:n]
        return x[n] - (w.real ** 2 + w.imag ** 2)

    def cons_jac(x):
        w = T + M @ x[:n]
        J = np.empty((len(z), n + 1))
        J[:, :n] = -2.0 * (w.real[:, None] * Mr + w.imag[:, None] * Mi)
        J[:, n] = 1.0
        return J

    x0 = np.zeros(n + 1)
    x0[n] = float(np.max(np.abs(T) ** 2))
    res = minimize(lambda x: x[n], x0, jac=lambda x: np.eye(n + 1)[n], method="SLSQP",
                   constraints=[{"type": "ineq", "fun": cons, "jac": cons_jac}],
                   options={"ftol": 1e-15, "maxiter": 500})
    x = res.x
    w = T + M @ x[:n]
    return float(np.max(np.abs(w) ** 2)), x[:n] / R ** (p + 1 + np.arange(n))


def optimize(sigma: np.ndarray, E: int, p: int = 2, rel_tol: float = 1e-7, tol: float = 1e-10):
    """(dt_max, alpha[0..E]) of Eq. OptimizationProblem for the eigenvalues sigma."""
    sigma = np.asarray(sigma, dtype=complex)
    sigma = sigma[np.abs(sigma) > 0]
    lam = np.abs(sigma).max()
    taylor = [1.0 / math.factorial(i) for i in range(p + 1)]
    if E <= p:
        raise ValueError("need E > p")

    def feasible(dt):
        v, alpha = _min_max_modulus(dt * sigma, E, p)
        return (alpha if v <= (1.0 + tol) ** 2 else None)

    lo, best, hi = 0.0, None, None
    dt = 1e-3 / lam
    while hi is None:
        a = feasible(dt)
        if a is None:
            hi = dt
        else:
            lo, best = dt, a
            dt *= 2.0
            if dt > 8.0 * E * E / lam:
                hi = dt
    if best is None:
        return 0.0, None
    while hi - lo > rel_tol * lo:
        mid = 0.5 * (lo + hi)
        a = feasible(mid)
        if a is None:
            hi = mid
        else:
            lo, best = mid, a
    return lo, np.concatenate([taylor, best])


def max_stable_dt(alpha: np.ndarray, sigma: np.ndarray, rel_tol: float = 1e-9, tol: float = 1e-10) -> float:
    """Largest dt with |P(dt lambda)| <= 1 + tol on sigma for the polynomial with coefficients alpha
    (bisection, starting from a stable small dt)."""
    sigma = np.asarray(sigma, dtype=complex)
    sigma = sigma[np.abs(sigma) > 0]
    lam = np.abs(sigma).max()
    ok = lambda dt: np.max(np.abs(np.polyval(np.asarray(alpha)[::-1], dt * sigma))) <= 1.0 + tol
    lo, hi = 0.0, 1e-3 / lam
    while ok(hi):
        lo, hi = hi, 2.0 * hi
        if hi > 1e3 * len(alpha) ** 2 / lam:
            return lo
    while hi - lo > rel_tol * hi:
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if ok(mid) else (lo, mid)
    return lo


def perk2_family_from_spectrum(sigma: np.ndarray, E: Sequence[int], S: int | None = None,
                               level_ratio: float = 2.0):
    """(c[S], a[R, S], dt_member[R], dt_family) of a second-order family for a quadtree whose
    finest level has the spectrum sigma.  Member r (E ascending) integrates the cells R-1-r
    levels coarser than the finest, whose spectrum is sigma / level_ratio^(R-1-r); its
    polynomial of degree E[r] is optimised for that spectrum.  dt_member[r] is its largest
    stable dt, dt_family the smallest of them (the step of the whole family)."""
    from . import perk2_disk_tableau, perk2_member

    E = [int(e) for e in E]
    S = int(S or max(E))
    R = len(E)
    c, _ = perk2_disk_tableau(E, S)
    rows, dts = [], []
    for r, e in enumerate(E):
        dt, alpha = optimize(np.asarray(sigma) / level_ratio ** (R - 1 - r), e, 2)
        rows.append(perk2_member(S, e, alpha))
        dts.append(dt)
    return c, np.array(rows), np.array(dts), float(min(dts))
