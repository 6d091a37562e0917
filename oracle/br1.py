"""BR1 viscous terms of the compressible Navier-Stokes equations (oracle; test infrastructure only).

The paper's viscous cases discretise the Navier-Stokes equations with DGSEM
and the BR1 scheme of Bassi and Rebay (cited in Sec. 7.1; stable for the
compressible equations by Gassner et al. 2018).  BR1 in strong form on an
element of size h:

1. gradient variables w = (v1, v2, T) with T = p / rho (gas constant 1);
2. lifting: q_d = (2/h) [ D_d w + (1/w_N) delta_N (w* - w) - (1/w_0) delta_0 (w* - w) ]
   with the central value w* = (w_L + w_R)/2 at every face node;
3. viscous flux f_v(u, q): stress tau_xx = mu (4/3 dv1/dx - 2/3 dv2/dy),
   tau_yy = mu (4/3 dv2/dy - 2/3 dv1/dx), tau_xy = mu (dv1/dy + dv2/dx),
   heat flux -kappa grad T, kappa = mu gamma / ((gamma - 1) Pr):
   f_v,x = (0, tau_xx, tau_xy, v1 tau_xx + v2 tau_xy + kappa dT/dx), likewise y;
4. divergence: du/dt += (2/h) [ D_d f_v,d + (1/w_N) delta_N (f* - f_v,d) - (1/w_0) delta_0 (f* - f_v,d) ]
   with the central flux f* = (f_v,L + f_v,R)/2 in the face's normal direction.

At a 2:1 hanging face the small side averages with the large side's nodal
values (of w, then of f_v) interpolated to its nodes; the large side takes the
L2 projection of the two half-face averages.  Every element's gradient is
computed from the full stage state, so the partitioned RHS is again the mask
of the full one.
"""

from __future__ import annotations

from collections import defaultdict

import numpy as np

from .dgsem import DGSEM
from .lgl import l2_project_two_halves, lagrange_eval


class NavierStokesDGSEM(DGSEM):
    def __init__(self, mesh, N: int = 3, surface_flux: str = "hll", gamma: float = 1.4, mu: float = 1e-3,
                 prandtl: float = 0.72, chunk: int = 4096):
        super().__init__(mesh, N, surface_flux, gamma, chunk)
        self.mu = mu
        self.kappa = mu * gamma / ((gamma - 1.0) * prandtl)

    def gradient_variables(self, V):
        rho = V[0]
        v1, v2 = V[1] / rho, V[2] / rho
        p = (self.gamma - 1.0) * (V[3] - 0.5 * rho * (v1 * v1 + v2 * v2))
        return np.stack([v1, v2, p / rho])

    def _face_averages(self, W):
        """Central face values of the nodal field W [nv, e, j, i] at every element face: dict (e, face) -> [nv, n]."""
        N = self.N
        x = self.x

        def trace(e, face):
            return (W[:, e, :, 0], W[:, e, :, N], W[:, e, 0, :], W[:, e, N, :])[face]

        out = {}
        for (A, B, d) in self.mesh.conforming:
            avg = 0.5 * (trace(A, 2 * d + 1) + trace(B, 2 * d))
            out[(A, 2 * d + 1)] = avg
            out[(B, 2 * d)] = avg
        halves = defaultdict(dict)
        for (A, B, d, large, half) in self.mesh.hanging:
            small, sface, lface = (B, 2 * d, 2 * d + 1) if large == A else (A, 2 * d + 1, 2 * d)
            s = 0.5 * (x - 1.0) if half == 0 else 0.5 * (x + 1.0)
            avg = 0.5 * (trace(small, sface) + lagrange_eval(x, trace(large, lface), s))
            out[(small, sface)] = avg
            halves[(large, lface)][half] = avg
        for key, hv in halves.items():
            out[key] = l2_project_two_halves(x, hv[0], hv[1])
        return out

    def _strong_derivative(self, F, Fstar, direction):
        """(2/h) [ D F + lifting of (F* - F) ] along x (direction 0) or y (1); F [nv, e, j, i]."""
        N = self.N
        w0, wN = self.w[0], self.w[N]
        if direction == 0:
            G = np.einsum("im,vejm->veji", self.D, F)
        else:
            G = np.einsum("jm,vemi->veji", self.D, F)
        for e in range(F.shape[1]):
            if direction == 0:
                G[:, e, :, N] += (Fstar[(e, 1)] - F[:, e, :, N]) / wN
                G[:, e, :, 0] -= (Fstar[(e, 0)] - F[:, e, :, 0]) / w0
            else:
                G[:, e, N, :] += (Fstar[(e, 3)] - F[:, e, N, :]) / wN
                G[:, e, 0, :] -= (Fstar[(e, 2)] - F[:, e, 0, :]) / w0
        return (2.0 / self.mesh.h)[None, :, None, None] * G

    def gradients(self, V):
        W = self.gradient_variables(V)
        Ws = self._face_averages(W)
        return self._strong_derivative(W, Ws, 0), self._strong_derivative(W, Ws, 1)

    def viscous_fluxes(self, V, qx, qy):
        rho = V[0]
        v1, v2 = V[1] / rho, V[2] / rho
        mu, k = self.mu, self.kappa
        dv1x, dv2x, dTx = qx
        dv1y, dv2y, dTy = qy
        txx = mu * (4.0 / 3.0 * dv1x - 2.0 / 3.0 * dv2y)
        tyy = mu * (4.0 / 3.0 * dv2y - 2.0 / 3.0 * dv1x)
        txy = mu * (dv1y + dv2x)
        z = np.zeros_like(txx)
        fx = np.stack([z, txx, txy, v1 * txx + v2 * txy + k * dTx])
        fy = np.stack([z, txy, tyy, v1 * txy + v2 * tyy + k * dTy])
        return fx, fy

    def viscous_rhs(self, U: np.ndarray) -> np.ndarray:
        V = np.moveaxis(np.asarray(U, dtype=np.float64), 1, 0)
        qx, qy = self.gradients(V)
        fx, fy = self.viscous_fluxes(V, qx, qy)
        fxs = self._face_averages(fx)
        fys = self._face_averages(fy)
        K = self._strong_derivative(fx, fxs, 0) + self._strong_derivative(fy, fys, 1)
        return np.ascontiguousarray(np.moveaxis(K, 0, 1))

    def rhs(self, U: np.ndarray) -> np.ndarray:
        return super().rhs(U) + self.viscous_rhs(U)
