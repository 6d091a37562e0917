"""Derivatives of the DGSEM right-hand side and of the P-ERK step (oracle; test infrastructure only).

The discrete adjoint of the library (Jacobian-vector and vector-Jacobian
products of the partitioned RHS, and the reverse sweep of one P-ERK step) is
checked against reverse- and forward-mode automatic differentiation of a
PyTorch (CPU, float64) transcription of the oracle's RHS in ``dgsem.py``.  The
transcription is the same definition written with torch operations so that
autograd applies; its value is pinned to the numpy oracle in the tests.
"""

from __future__ import annotations

from collections import defaultdict

import numpy as np
import torch

from .lgl import derivative_matrix, l2_project_two_halves, lagrange_basis, lgl_nodes_weights
from .perk import PERKFamily
from .treemesh import TreeMesh

GAMMA = 1.4


def _prim(u, g):
    rho = u[0]
    v1 = u[1] / rho
    v2 = u[2] / rho
    p = (g - 1.0) * (u[3] - 0.5 * rho * (v1 * v1 + v2 * v2))
    return rho, v1, v2, p


def _phys(u, d, g):
    rho, v1, v2, p = _prim(u, g)
    vn = v1 if d == 0 else v2
    z = torch.zeros_like(p)
    return torch.stack([rho * vn, u[1] * vn + (p if d == 0 else z), u[2] * vn + (p if d == 1 else z), (u[3] + p) * vn])


def _log_mean(a, b):
    # as euler.log_mean: the artanh series for |f| < 1e-2 (smooth across a == b), log1p otherwise
    d = b - a
    s = a + b
    f = d / s
    u = f * f
    small = torch.abs(f) < 1e-2
    series = s / (2.0 * (1.0 + u / 3.0 + u * u / 5.0 + u * u * u / 7.0))
    safe = torch.where(small, torch.ones_like(d), d)
    return torch.where(small, series, safe / torch.log1p(safe / a))


def ec_flux(uL, uR, d, g=GAMMA):
    rL, v1L, v2L, pL = _prim(uL, g)
    rR, v1R, v2R, pR = _prim(uR, g)
    rho_ln = _log_mean(rL, rR)
    beta_ln = _log_mean(rL / pL, rR / pR)
    v1m, v2m, pm = 0.5 * (v1L + v1R), 0.5 * (v2L + v2R), 0.5 * (pL + pR)
    vnL, vnR = (v1L, v1R) if d == 0 else (v2L, v2R)
    f_rho = rho_ln * 0.5 * (vnL + vnR)
    z = torch.zeros_like(pm)
    return torch.stack([f_rho, f_rho * v1m + (pm if d == 0 else z), f_rho * v2m + (pm if d == 1 else z),
                        f_rho * (0.5 * (v1L * v1R + v2L * v2R) + 1.0 / ((g - 1.0) * beta_ln))
                        + 0.5 * (pL * vnR + pR * vnL)])


def _speeds(uL, uR, d, g):
    rL, v1L, v2L, pL = _prim(uL, g)
    rR, v1R, v2R, pR = _prim(uR, g)
    vL, vR = (v1L, v1R) if d == 0 else (v2L, v2R)
    cL, cR = torch.sqrt(g * pL / rL), torch.sqrt(g * pR / rR)
    return torch.minimum(vL - cL, vR - cR), torch.maximum(vL + cL, vR + cR)


def hll_flux(uL, uR, d, g=GAMMA):
    SL, SR = _speeds(uL, uR, d, g)
    fL, fR = _phys(uL, d, g), _phys(uR, d, g)
    mid = (SR * fL - SL * fR + SL * SR * (uR - uL)) / (SR - SL)
    return torch.where(SL >= 0.0, fL, torch.where(SR <= 0.0, fR, mid))


def hllc_flux(uL, uR, d, g=GAMMA):
    SL, SR = _speeds(uL, uR, d, g)
    rL, v1L, v2L, pL = _prim(uL, g)
    rR, v1R, v2R, pR = _prim(uR, g)
    vL, tL = (v1L, v2L) if d == 0 else (v2L, v1L)
    vR, tR = (v1R, v2R) if d == 0 else (v2R, v1R)
    Ss = (pR - pL + rL * vL * (SL - vL) - rR * vR * (SR - vR)) / (rL * (SL - vL) - rR * (SR - vR))
    fL, fR = _phys(uL, d, g), _phys(uR, d, g)

    def star(r, v, t, p, E, S):
        fac = r * (S - v) / (S - Ss)
        Es = fac * (E / r + (Ss - v) * (Ss + p / (r * (S - v))))
        return torch.stack([fac, fac * Ss, fac * t, Es]) if d == 0 else torch.stack([fac, fac * t, fac * Ss, Es])

    fLs = fL + SL * (star(rL, vL, tL, pL, uL[3], SL) - uL)
    fRs = fR + SR * (star(rR, vR, tR, pR, uR[3], SR) - uR)
    return torch.where(SL >= 0.0, fL, torch.where(Ss >= 0.0, fLs, torch.where(SR > 0.0, fRs, fR)))


FLUXES = {"hll": hll_flux, "hllc": hllc_flux, "ec": ec_flux}


class TorchDGSEM:
    """The oracle's strong-form flux-differencing DGSEM written with torch operations."""

    def __init__(self, mesh: TreeMesh, N: int = 3, surface_flux: str = "hll", gamma: float = GAMMA):
        self.mesh = mesh
        self.N = N
        self.g = gamma
        x, w = lgl_nodes_weights(N)
        self.x = x
        self.w = w
        self.D2 = torch.tensor(2.0 * derivative_matrix(x))
        self.fstar = FLUXES[surface_flux]
        self.h = torch.tensor(mesh.h)
        # large-trace evaluation at the small-face nodes, and the half-face L2 projections
        self.P = [torch.tensor(lagrange_basis(x, 0.5 * (x - 1.0))), torch.tensor(lagrange_basis(x, 0.5 * (x + 1.0)))]
        n = N + 1
        R = []
        for half in (0, 1):
            cols = []
            for k in range(n):
                e = np.zeros(n)
                e[k] = 1.0
                z = np.zeros(n)
                cols.append(l2_project_two_halves(x, e, z) if half == 0 else l2_project_two_halves(x, z, e))
            R.append(torch.tensor(np.stack(cols, axis=1)))     # phi = R_half @ f_half
        self.R = R

    def rhs(self, U: torch.Tensor) -> torch.Tensor:
        N, g = self.N, self.g
        V = U.movedim(1, 0)                                            # [4, e, j, i]
        Fx = ec_flux(V[:, :, :, :, None], V[:, :, :, None, :], 0, g)
        Fy = ec_flux(V[:, :, :, None, :], V[:, :, None, :, :], 1, g)
        vol = torch.einsum("im,vejim->veji", self.D2, Fx) + torch.einsum("jm,vejmi->veji", self.D2, Fy)

        def trace(e, face):
            return (V[:, e, :, 0], V[:, e, :, N], V[:, e, 0, :], V[:, e, N, :])[face]

        Fs = {}
        for (A, B, d) in self.mesh.conforming:
            f = self.fstar(trace(A, 2 * d + 1), trace(B, 2 * d), d, g)
            Fs[(A, 2 * d + 1)] = f
            Fs[(B, 2 * d)] = f
        halves = defaultdict(dict)
        for (A, B, d, large, half) in self.mesh.hanging:
            small, sface, lface = (B, 2 * d, 2 * d + 1) if large == A else (A, 2 * d + 1, 2 * d)
            ul = trace(large, lface) @ self.P[half].T
            us = trace(small, sface)
            f = self.fstar(ul, us, d, g) if large == A else self.fstar(us, ul, d, g)
            Fs[(small, sface)] = f
            halves[(large, lface)][half] = f
        for key, hv in halves.items():
            Fs[key] = hv[0] @ self.R[0].T + hv[1] @ self.R[1].T
        w0, wN = float(self.w[0]), float(self.w[N])
        Sl = []
        for e in range(V.shape[1]):
            s = torch.zeros_like(V[:, e])
            s[:, :, 0] = s[:, :, 0] - (Fs[(e, 0)] - _phys(V[:, e, :, 0], 0, g)) / w0
            s[:, :, N] = s[:, :, N] + (Fs[(e, 1)] - _phys(V[:, e, :, N], 0, g)) / wN
            s[:, 0, :] = s[:, 0, :] - (Fs[(e, 2)] - _phys(V[:, e, 0, :], 1, g)) / w0
            s[:, N, :] = s[:, N, :] + (Fs[(e, 3)] - _phys(V[:, e, N, :], 1, g)) / wN
            Sl.append(s)
        S = torch.stack(Sl, dim=1)
        K = -(2.0 / self.h)[None, :, None, None] * (vol + S)
        return K.movedim(0, 1)


def vjp_rhs(dg: TorchDGSEM, U: np.ndarray, lam: np.ndarray, active=None) -> np.ndarray:
    """(dF/dU)^T lam, F masked to ``active`` elements when given."""
    Ut = torch.tensor(U, requires_grad=True)
    K = dg.rhs(Ut)
    if active is not None:
        K = K * torch.tensor(np.asarray(active, dtype=np.float64))[:, None, None, None]
    (g,) = torch.autograd.grad(K, Ut, torch.tensor(lam))
    return g.numpy()


def jvp_rhs(dg: TorchDGSEM, U: np.ndarray, v: np.ndarray) -> np.ndarray:
    """(dF/dU) v by forward-mode differentiation."""
    _, t = torch.func.jvp(dg.rhs, (torch.tensor(U),), (torch.tensor(v),))
    return t.numpy()


def perk_step_torch(dg: TorchDGSEM, U: torch.Tensor, dt: float, fam: PERKFamily, method) -> torch.Tensor:
    """The dense partitioned RK step (as in perk.prkm_step) with torch operations."""
    coef = torch.tensor(np.stack(fam.A))[torch.tensor(method)]          # [e, S, S]
    K = []
    for i in range(fam.S):
        Y = U
        for j in range(i):
            a = coef[:, i, j]
            if torch.any(a != 0):
                Y = Y + dt * a[:, None, None, None] * K[j]
        K.append(dg.rhs(Y))
    Un = U
    for i in range(fam.S):
        if fam.b[i] != 0.0:
            Un = Un + dt * float(fam.b[i]) * K[i]
    return Un


def vjp_steps(dg: TorchDGSEM, U0: np.ndarray, lam: np.ndarray, dt: float, fam: PERKFamily, method,
              n_steps: int) -> np.ndarray:
    """(dU_n / dU_0)^T lam for n P-ERK steps from U_0."""
    Ut = torch.tensor(U0, requires_grad=True)
    U = Ut
    for _ in range(n_steps):
        U = perk_step_torch(dg, U, dt, fam, method)
    (g,) = torch.autograd.grad(U, Ut, torch.tensor(lam))
    return g.numpy()
