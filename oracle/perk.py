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


def perk2_abscissae(S: int) -> np.ndarray:
    return np.arange(S, dtype=np.float64) / (2.0 * (S - 1))


def perk2_free_coefficients(S: int, E: int, alpha: Sequence[float]) -> np.ndarray:
    """a_{i,i-1} for i = 1..S (entries 0 where the member has no such entry),
    from alpha_3..alpha_E by Eq. PERKCoeffsConstruction:
        a_{S-i} = alpha_{3+i} / (c_{S-i-1} prod_{j=0}^{i-1} a_{S-j}),  i = 0, ..., E-3.
    Returned array is indexed by the 1-based stage number (index 0 unused)."""
    c = np.concatenate([[np.nan], perk2_abscissae(S)])   # 1-based c
    a = np.zeros(S + 1)
    for i in range(0, E - 2):
        prod = 1.0
        for j in range(i):
            prod *= a[S - j]
        a[S - i] = alpha[3 + i] / (c[S - i - 1] * prod)
    return a


@dataclass
class PERKFamily:
    S: int
    E: List[int]                 # ascending stage evaluations, member r = 1..R
    c: np.ndarray                # [S]
    b: np.ndarray                # [S]
    A: List[np.ndarray]          # R dense S x S Butcher arrays
    order: int = 2

    @property
    def R(self) -> int:
        return len(self.E)

    def active(self, r: int, i: int) -> bool:
        """Whether member r (0-based) evaluates stage i (0-based): K_1 always,
        otherwise stages S-E+2 .. S (1-based)."""
        return i == 0 or (i + 1) >= self.S - self.E[r] + 2


def perk2_family(E_list: Sequence[int], S: int | None = None, alphas=None) -> PERKFamily:
    """Second-order P-ERK family with members E_list (ascending) and S = max(E) stages."""
    E_list = [int(e) for e in E_list]
    S = S or max(E_list)
    c = perk2_abscissae(S)
    b = np.zeros(S)
    b[-1] = 1.0
    A = []
    for r, E in enumerate(E_list):
        alpha = disk_polynomial_alpha(E) if alphas is None else np.asarray(alphas[r])
        a_free = perk2_free_coefficients(S, E, alpha)
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
                Y = Y + dt * a_e[:, None, None, None] * K[j]
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
    Eq. CFL_DG summed over both directions)."""
    rho = U[:, 0]
    v1 = U[:, 1] / rho
    v2 = U[:, 2] / rho
    p = (gamma - 1.0) * (U[:, 3] - 0.5 * rho * (v1 * v1 + v2 * v2))
    c = np.sqrt(gamma * p / rho)
    lam = (np.abs(v1) + np.abs(v2) + 2.0 * c).reshape(len(h), -1).max(axis=1)
    return float(cfl * np.min(h / ((N + 1) * lam)))
