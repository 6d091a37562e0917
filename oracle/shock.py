"""Subcell shock capturing of the DGSEM volume term (oracle; test infrastructure only).

The paper's hyperbolic runs (Sec. 7.2) blend the flux-differencing volume term with a
first-order finite-volume term on the LGL subcells of each element (Hennemann, Rueda-Ramirez,
Hindenlang and Gassner, J. Comput. Phys. 2021), element by element:

1. Indicator.  epsilon = rho p at the nodes (Hennemann et al.'s variable; the paper's KH run
   bases it on the density, epsilon = rho, Sec. 7.2.1), written in the orthonormal Legendre basis
   (modes a along x, b along y): m = V^{-1} epsilon V^{-T}, V_ik = L_k(x_i).  With
   E_k = sum_{max(a,b) <= k} m_ab^2, the share of the highest modes is
       energy = max((E_N - E_{N-1}) / E_N, (E_{N-1} - E_{N-2}) / E_{N-1}).
   Threshold T = 0.5 * 10^(-1.8 (N+1)^(1/4)), sharpness s = ln((1 - 1e-4) / 1e-4):
       alpha = 1 / (1 + exp(-(s / T) (energy - T))),
   set to 0 below alpha_min = 1e-3 and capped at alpha_max (0.5 by default).
2. Finite-volume term.  Along each grid line of the element the LGL node i owns a subcell of
   reference width w_i (the weights sum to the reference length 2).  With the numerical flux
   F_{i+1/2} = f*(u_i, u_{i+1}) between neighbouring nodes (i = 0 .. N-1) and the physical flux
   at the element ends, F_{-1/2} = f(u_0), F_{N+1/2} = f(u_N) (the rest of the face flux stays in
   the surface term of the strong form), the term is (F_{i+1/2} - F_{i-1/2}) / w_i.  Like the
   flux-differencing term it sums, with the weights, to f(u_N) - f(u_0), so the blend keeps the
   scheme conservative.
3. Blend.  volume = (1 - alpha) (sum_m 2 D_im f#(u_i, u_m) + ...) + alpha (finite-volume term),
   in both directions; the surface term of the strong form is unchanged.
"""

from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import legendre as npleg

from . import euler
from .br1 import NavierStokesDGSEM
from .dgsem import DGSEM

ALPHA_MIN = 1e-3
ALPHA_MAX = 0.5


def legendre_vandermonde(x: np.ndarray) -> np.ndarray:
    """V_ik = L_k(x_i), L_k the orthonormal Legendre polynomials on [-1, 1]."""
    n = len(x)
    V = np.empty((n, n))
    for k in range(n):
        c = np.zeros(k + 1)
        c[k] = 1.0
        V[:, k] = npleg.legval(x, c) * math.sqrt(k + 0.5)
    return V


def blending_factor(U: np.ndarray, x: np.ndarray, gamma: float = euler.GAMMA,
                    alpha_max: float = ALPHA_MAX, variable: str = "density_pressure") -> np.ndarray:
    """alpha per element of the nodal state U [e, 4, j, i] (step 1 above); variable is
    "density_pressure" (epsilon = rho p) or "density" (epsilon = rho)."""
    N = len(x) - 1
    rho, _, _, p = euler.primitives(np.moveaxis(U, 1, 0), gamma)
    eps = rho * p if variable == "density_pressure" else rho        # [e, j, i]
    Vinv = np.linalg.inv(legendre_vandermonde(x))
    m = np.einsum("bj,eji,ai->eba", Vinv, eps, Vinv)                # modes [e, b, a]
    a_idx = np.arange(N + 1)
    order = np.maximum(a_idx[None, :], a_idx[:, None])              # max(a, b) for [b, a]
    m2 = m * m

    def E(k):
        return np.sum(np.where(order <= k, m2, 0.0), axis=(1, 2))

    EN, EN1, EN2 = E(N), E(N - 1), E(N - 2)
    energy = np.maximum((EN - EN1) / EN, (EN1 - EN2) / EN1)
    T = 0.5 * 10.0 ** (-1.8 * (N + 1) ** 0.25)
    s = math.log((1.0 - 1e-4) / 1e-4)
    alpha = 1.0 / (1.0 + np.exp(-(s / T) * (energy - T)))
    alpha = np.where(alpha < ALPHA_MIN, 0.0, alpha)
    return np.minimum(alpha, alpha_max)


def finite_volume_term(V: np.ndarray, w: np.ndarray, fstar, gamma: float = euler.GAMMA) -> np.ndarray:
    """The subcell finite-volume term (step 2) in x plus in y; V = [4, e, j, i]."""
    N = len(w) - 1
    out = np.zeros_like(V)
    for d in (0, 1):
        W = V if d == 0 else np.swapaxes(V, 2, 3)                  # lines along the last axis
        F = np.empty(W.shape[:3] + (N + 2,))                         # [4, e, line, N + 2]
        F[..., 0] = euler.physical_flux(W[..., 0], d, gamma)
        F[..., N + 1] = euler.physical_flux(W[..., N], d, gamma)
        for i in range(N):
            F[..., i + 1] = fstar(W[..., i], W[..., i + 1], d, gamma)
        T = (F[..., 1:] - F[..., :-1]) / w
        out += T if d == 0 else np.swapaxes(T, 2, 3)
    return out


def blended_volume(dg: DGSEM, V: np.ndarray, alpha_max: float, variable: str) -> np.ndarray:
    """Step 3 for the scheme dg (its flux-differencing volume term, nodes, weights and surface
    flux); V = [4, e, j, i]."""
    vol = DGSEM._volume(dg, V)
    alpha = blending_factor(np.moveaxis(V, 0, 1), dg.x, dg.gamma, alpha_max, variable)
    fv = finite_volume_term(V, dg.w, dg.fstar, dg.gamma)
    a = alpha[None, :, None, None]
    return (1.0 - a) * vol + a * fv


class ShockCapturingDGSEM(DGSEM):
    """The DGSEM of dgsem.py with the blended volume term (steps 1-3); the subcells use the
    surface flux of the scheme."""

    def __init__(self, mesh, N: int = 3, surface_flux: str = "hlle", gamma: float = euler.GAMMA,
                 alpha_max: float = ALPHA_MAX, variable: str = "density_pressure", chunk: int = 4096):
        super().__init__(mesh, N, surface_flux, gamma, chunk)
        self.alpha_max = alpha_max
        self.variable = variable

    def _volume(self, V: np.ndarray) -> np.ndarray:
        return blended_volume(self, V, self.alpha_max, self.variable)


class ShockCapturingNavierStokesDGSEM(NavierStokesDGSEM):
    """The Navier-Stokes DGSEM of br1.py with the blended inviscid volume term."""

    def __init__(self, mesh, N: int = 3, surface_flux: str = "hlle", gamma: float = euler.GAMMA, mu: float = 1e-3,
                 prandtl: float = 0.72, alpha_max: float = ALPHA_MAX, variable: str = "density_pressure"):
        super().__init__(mesh, N, surface_flux, gamma, mu, prandtl)
        self.alpha_max = alpha_max
        self.variable = variable

    def _volume(self, V: np.ndarray) -> np.ndarray:
        return blended_volume(self, V, self.alpha_max, self.variable)
