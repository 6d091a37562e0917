"""P-ERK coefficient construction and the dense partitioned RK step (oracle; test infrastructure only).

Second-order P-ERK (Sec. 3.1, Eq. PERK_ButcherTableauClassic; Sec. 4.3.1):
  * S stages with shared abscissae c_i = (i - 1) / (2 (S - 1)) and weights b = e_S.
  * A member with E evaluations computes K_1 and K_{S-E+2}, ..., K_S; its only
    non-zero Butcher entries are a_{i,i-1} for i = S-E+3 .. S (free) and
    a_{i,1} = c_i - a_{i,i-1} (internal consistency, Eq. InternalConsistency).
  * The free entries follow from the stability polynomial's monomial
    coefficients alpha_3 .. alpha_E by the sequential recursion of
    Eq. PERKCoeffsConstruction, read with i = 0 .. E-3.

The step is the partitioned Runge-Kutta method in Butcher form
(Eq. PartitionedRKSystem) with the mask matrices of Sec. 2.2, evaluated
densely: every stage K_j = F(Y_j) is computed on every element and the full
S x S arrays A^(r) decide what enters Y_i:

  Y_i = U_n + dt sum_j sum_r a_ij^(r) I^(r) K_j,     U_{n+1} = U_n + dt sum_i b_i K_i.
"""

from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Callable, List, Sequence

import numpy as np


def disk_polynomial_alpha(E: int) -> np.ndarray:
    """Monomial coefficients of P_{2;E}(z) = 1/E + ((E-1)/E) (1 + z/(E-1))^E.

    This degree-E, second-order polynomial is stable on the disk
    |z + (E-1)| <= E-1, the spectrum of the first-order upwind scheme that the
    paper's Sec. 3.2.2 says has an analytically known optimum; returns
    alpha[0..E] (alpha_0 = 1, alpha_1 = 1, alpha_2 = 1/2).
    """
    r = E - 1.0
    alpha = np.array([(r / E) * math.comb(E, k) / r ** k for k in range(E + 1)])
    alpha[0] += 1.0 / E
    return alpha


def perk2_abscissae(S: int, b_S: float = 1.0) -> np.ndarray:
    """c_i = c_S (i - 1)/(S - 1) with c_S = 1/(2 b_S): 1/2 for the weights b = e_S of
    Eq. PERK_ButcherTableauClassic; the variants of Sec. 3.1 with b_1 = 1 - b_S take
    c_S = 1 (Heun, b_S = 1/2) and c_S = 2/3 (Ralston, b_S = 3/4)."""
    return np.arange(S, dtype=np.float64) / (2.0 * b_S * (S - 1))


def perk2_free_coefficients(S: int, E: int, alpha: Sequence[float], b_S: float = 1.0) -> np.ndarray:
    """a_{i,i-1} for i = 1..S (entries 0 where the member has no such entry),
    from alpha_3..alpha_E by Eq. PERKCoeffsConstruction:
        a_{S-i} = alpha_{3+i} / (b_S c_{S-i-1} prod_{j=0}^{i-1} a_{S-j}),  i = 0, ..., E-3.
    (The coefficient of z^k, k >= 2, of 1 + z b^T (I - zA)^{-1} 1 is b^T A^{k-1} 1, and only
    b_S contributes because the first row of A is zero.)
    Returned array is indexed by the 1-based stage number (index 0 unused)."""
    c = np.concatenate([[np.nan], perk2_abscissae(S, b_S)])   # 1-based c
    a = np.zeros(S + 1)
    for i in range(0, E - 2):
        prod = 1.0
        for j in range(i):
            prod *= a[S - j]
        a[S - i] = alpha[3 + i] / (b_S * c[S - i - 1] * prod)
    return a


@dataclass
class PERKFamily:
    S: int
    E: List[int]                 # ascending stage evaluations, member r = 1..R
    c: np.ndarray                # [S]
    b: np.ndarray                # [S]
    A: List[np.ndarray]          # R dense S x S Butcher arrays
    order: int = 2
    evaluated: List[List[int]] | None = None   # per member, the 1-based stages it evaluates

    @property
    def R(self) -> int:
        return len(self.E)

    def active(self, r: int, i: int) -> bool:
        """Whether member r (0-based) evaluates stage i (0-based): K_1 always, otherwise
        stages S-E+2 .. S (1-based) in the classic pattern, or the pattern's stages."""
        if self.evaluated is not None:
            return (i + 1) in self.evaluated[r]
        return i == 0 or (i + 1) >= self.S - self.E[r] + 2


def pattern_stages(S: int, E: int, pattern: str) -> List[int]:
    """The 1-based stages a member with E evaluations computes in an S-stage family.
    classic (Eq. PERK_ButcherTableauClassic): 1 and S-E+2 .. S; early (shared evaluations
    first, Eq. PERK_ButcherTableauEarlyShared): 1 .. E-1 and S; alternating
    (Eq. PERK_ButcherTableauAlternating): 1 and s_k = S - floor((E-1-k)(S-1)/(E-1) + 1/2),
    k = 1 .. E-1, which spreads the evaluations evenly (S = 6, E = 4: 1, 3, 4, 6 as printed)."""
    if E == S or pattern == "classic":
        return [1] + list(range(S - E + 2, S + 1))
    if pattern == "early":
        return list(range(1, E)) + [S]
    if pattern == "alternating":
        return [1] + [S - math.floor((E - 1 - k) * (S - 1) / (E - 1) + 0.5) for k in range(1, E)]
    raise ValueError(pattern)


def pattern_member(S: int, E: int, alpha: Sequence[float], pattern: str, b_S: float = 1.0) -> np.ndarray:
    """Dense S x S array of a second-order member with stage pattern `pattern`: every evaluated
    stage after the first one past K_1 couples to the previous evaluated stage, s_k -> s_{k-1}
    (k >= 2), the rest of its abscissa on K_1 (internal consistency).  With b = (1 - b_S) e_1 +
    b_S e_S the coefficient of z^{3+j} of the stability polynomial is
    b_S c_{s_{E-2-j}} prod_{q=0}^{j} a_{s_{E-1-q}, s_{E-2-q}}, which gives the couplings from
    alpha_3 .. alpha_E one after the other, from the last stage backwards (the recursion of
    Eq. PERKCoeffsConstruction along the member's own stages)."""
    c = perk2_abscissae(S, b_S)
    st = pattern_stages(S, E, pattern)                   # s_0 = 1 < s_1 < ... < s_{E-1} = S
    a = {}
    prod = 1.0
    for j in range(E - 2):
        hi, lo = st[E - 1 - j], st[E - 2 - j]
        v = alpha[3 + j] / (b_S * c[lo - 1] * prod)
        a[(hi, lo)] = v
        prod *= v
    M = np.zeros((S, S))
    for i1 in range(2, S + 1):
        src = [lo for (hi, lo) in a if hi == i1]
        ai = a[(i1, src[0])] if src else 0.0
        if src:
            M[i1 - 1, src[0] - 1] += ai
        M[i1 - 1, 0] += c[i1 - 1] - ai
    return M


def perk2_family(E_list: Sequence[int], S: int | None = None, alphas=None, b_S: float = 1.0,
                 pattern: str = "classic") -> PERKFamily:
    """Second-order P-ERK family with members E_list (ascending) and S = max(E) stages; weights
    b_1 = 1 - b_S, b_S (b_S = 1: Eq. PERK_ButcherTableauClassic); stage pattern classic,
    alternating or early (Sec. 3.2.4)."""
    E_list = [int(e) for e in E_list]
    S = S or max(E_list)
    c = perk2_abscissae(S, b_S)
    b = np.zeros(S)
    b[-1] = b_S
    b[0] += 1.0 - b_S
    if pattern != "classic":
        A = [pattern_member(S, E, disk_polynomial_alpha(E) if alphas is None else np.asarray(alphas[r]), pattern, b_S)
             for r, E in enumerate(E_list)]
        return PERKFamily(S=S, E=E_list, c=c, b=b, A=A, order=2,
                          evaluated=[pattern_stages(S, E, pattern) for E in E_list])
    A = []
    for r, E in enumerate(E_list):
        alpha = disk_polynomial_alpha(E) if alphas is None else np.asarray(alphas[r])
        a_free = perk2_free_coefficients(S, E, alpha, b_S)
        M = np.zeros((S, S))
        for i1 in range(2, S + 1):                 # 1-based stage number
            ai = a_free[i1]
            M[i1 - 1, i1 - 2] += ai
            M[i1 - 1, 0] += c[i1 - 1] - ai
        A.append(M)
    return PERKFamily(S=S, E=E_list, c=c, b=b, A=A, order=2)


def stability_polynomial(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Monomial coefficients of P(z) = 1 + z b^T (I - z A)^{-1} 1 = 1 + sum_k z^{k+1} b^T A^k 1
    (finite for explicit, i.e. strictly lower triangular, A)."""
    S = len(b)
    coeffs = [1.0]
    v = np.ones(S)
    for _ in range(S):
        coeffs.append(float(b @ v))
        v = A @ v
    return np.array(coeffs)


def element_methods(levels: np.ndarray, R: int) -> np.ndarray:
    """Member index (0-based) of every element: the finest present level gets
    member R-1, the next coarser R-2, ..., all remaining levels member 0
    (Sec. 6.4.1: the highest-evaluation method on the finest level, the lowest
    one for every level beyond the family's size)."""
    levels = np.asarray(levels)
    lmax = int(levels.max())
    return np.maximum(0, (R - 1) - (lmax - levels)).astype(np.int64)


def prkm_step(rhs: Callable[[np.ndarray], np.ndarray], U: np.ndarray, dt: float, fam: PERKFamily,
              method: np.ndarray) -> np.ndarray:
    """One step of Eq. PartitionedRKSystem with the dense arrays of ``fam``;
    ``method[e]`` is the member (0-based) that integrates element e."""
    S = fam.S
    K = []
    coef = np.stack([fam.A[r] for r in range(fam.R)])     # [R, S, S]
    for i in range(S):
        Y = U.copy()
        for j in range(i):
            a_e = coef[method, i, j]                       # a_ij^(r(e)) per element
            if np.any(a_e != 0.0):
                Y = Y + dt * a_e.reshape((-1,) + (1,) * (U.ndim - 1)) * K[j]
        K.append(rhs(Y))
    Un = U.copy()
    for i in range(S):
        if fam.b[i] != 0.0:
            Un = Un + dt * fam.b[i] * K[i]
    return Un


def rk_step(rhs: Callable[[np.ndarray], np.ndarray], U: np.ndarray, dt: float, A: np.ndarray,
            b: np.ndarray) -> np.ndarray:
    """Standard explicit Runge-Kutta step with Butcher array A and weights b."""
    K = []
    for i in range(len(b)):
        Y = U.copy()
        for j in range(i):
            if A[i, j] != 0.0:
                Y = Y + dt * A[i, j] * K[j]
        K.append(rhs(Y))
    return U + dt * sum(b[i] * K[i] for i in range(len(b)) if b[i] != 0.0)


def max_wave_speed_dt(U: np.ndarray, h: np.ndarray, N: int, cfl: float, gamma: float = 1.4) -> float:
    """dt = cfl * min_e h_e / ((N + 1) lambda_e), lambda_e = max over the
    element's nodes of |v1| + |v2| + 2c (the convective time scale of
    Eq. CFL_DG summed over both directions).  The sound speed, and with it the
    step, exists only for admissible states: NaN if any node has rho <= 0,
    p <= 0 or a non-finite entry."""
    rho = U[:, 0]
    with np.errstate(divide="ignore", invalid="ignore"):
        v1 = U[:, 1] / rho
        v2 = U[:, 2] / rho
        p = (gamma - 1.0) * (U[:, 3] - 0.5 * rho * (v1 * v1 + v2 * v2))
        if not (np.all(rho > 0.0) and np.all(p > 0.0)):
            return float("nan")
        c = np.sqrt(gamma * p / rho)
    lam = (np.abs(v1) + np.abs(v2) + 2.0 * c).reshape(len(h), -1).max(axis=1)
    return float(cfl * np.min(h / ((N + 1) * lam)))


# ---------------------------------------------------------------------------
# Third-order P-ERK (Sec. 3.3, Eq. PERK_ThirdOrderShuOsher and Eq. Free_Timesteps;
# Sec. 4.3.2): abscissae c_i = (i-1)/(S-3) for i <= S-2, c_{S-1} = 1, c_S = 1/2,
# weights b_1 = b_{S-1} = 1/6, b_S = 2/3.

def perk3_abscissae(S: int) -> np.ndarray:
    c = np.zeros(S)
    for i in range(1, S - 2):                       # 1-based i = 2 .. S-2 (none for S = 3)
        c[i] = i / (S - 3.0)
    c[S - 2] = 1.0
    c[S - 1] = 0.5
    return c


def perk3_weights(S: int) -> np.ndarray:
    b = np.zeros(S)
    b[0] = 1.0 / 6.0
    b[S - 2] += 1.0 / 6.0
    b[S - 1] += 2.0 / 3.0
    return b


def disk_polynomial3_alpha(E: int, tol: float = 1e-12):
    """Third-order polynomial of degree E stable on the largest disk |z + r| <= r
    among P(z) = sum_k d_k (1 + z/r)^k with d >= 0, sum d = 1 (then |P| <= 1 on
    the disk): the three order conditions P'(0) = P''(0) = P'''(0) = 1 are
    sum k d_k = r, sum k(k-1) d_k = r^2, sum k(k-1)(k-2) d_k = r^3; the largest
    r with a feasible d is found by bisection on a linear-programming feasibility
    test.  Returns (alpha[0..E], r)."""
    from scipy.optimize import linprog

    k = np.arange(E + 1, dtype=np.float64)

    Aeq = np.stack([np.ones_like(k), k, k * (k - 1), k * (k - 1) * (k - 2)])

    def feasible(r):
        beq = np.array([1.0, r, r * r, r ** 3])
        res = linprog(np.zeros(E + 1), A_eq=Aeq, b_eq=beq, bounds=[(0, None)] * (E + 1), method="highs")
        if res.status != 0:
            return None
        # the solver's own feasibility tolerance is ~1e-7; accept only solutions that hold to rounding
        d = np.maximum(res.x, 0.0)
        return d if np.max(np.abs(Aeq @ d - beq) / np.maximum(1.0, beq)) < 1e-12 else None

    lo, hi = 0.5, float(E)
    assert feasible(lo) is not None
    while hi - lo > tol * hi:
        mid = 0.5 * (lo + hi)
        if feasible(mid) is not None:
            lo = mid
        else:
            hi = mid
    d = feasible(lo)
    alpha = np.array([sum(d[j] * math.comb(j, m) for j in range(m, E + 1)) / lo ** m for m in range(E + 1)])
    return alpha, lo


def perk3_member(S: int, E: int, alpha, seeds: int = 16):
    """Free entries a_{i,i-1}, i = S-E+3..S, of a third-order member with E
    evaluations: the stability polynomial 1 + z b^T (I - z A)^{-1} 1 must have
    the coefficients alpha_3..alpha_E (alpha_3 = 1/6 is the coupling condition
    b_S a_S + b_{S-1} a_{S-1} = 1/6), with 0 < a_i < c_i (Sec. 4.3.2: a trust-region
    solve from seeded random starts; the first start that converges with all
    entries positive is taken).  Returns the dense S x S array."""
    from scipy.optimize import least_squares

    c = perk3_abscissae(S)
    b = perk3_weights(S)
    idx = list(range(S - E + 2, S))                  # 0-based stage rows with a free a_{i,i-1}

    def build(x):
        A = np.zeros((S, S))
        for i in range(1, S):
            A[i, 0] = c[i]
        for xi, i in zip(x, idx):
            A[i, i - 1] = xi
            A[i, 0] = c[i] - xi
        return A

    def residual(x):
        p = stability_polynomial(build(x), b)
        return (p[3:E + 1] - alpha[3:E + 1]) / alpha[3:E + 1]

    rng = np.random.default_rng(20240308)
    best = None
    for _ in range(seeds):
        x0 = rng.uniform(0.05, 0.95, len(idx)) * c[idx]
        res = least_squares(residual, x0, bounds=(np.zeros(len(idx)), c[idx]), xtol=1e-15, ftol=1e-15, gtol=1e-15)
        if np.max(np.abs(res.fun)) < 1e-10 and np.all(res.x > 0) and np.all(c[idx] - res.x > 0):
            best = res.x
            break
    if best is None:
        raise RuntimeError(f"no admissible third-order member for S={S}, E={E}")
    return build(best)


def perk3_family(E_list: Sequence[int], S: int | None = None) -> PERKFamily:
    E_list = [int(e) for e in E_list]
    S = S or max(E_list)
    A = [perk3_member(S, E, disk_polynomial3_alpha(E)[0]) for E in E_list]
    return PERKFamily(S=S, E=E_list, c=perk3_abscissae(S), b=perk3_weights(S), A=A, order=3)
