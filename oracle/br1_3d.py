"""BR1 viscous terms of the 3D compressible Navier-Stokes equations (oracle; test infrastructure only).

The paper's three-dimensional run (Sec. 7.1.3, the Taylor-Green vortex at Re 1600, Pr 0.72) is
viscous; its viscous terms are discretised with BR1 as in the 2D cases of Sec. 7.1 (``br1.py``),
here on hexahedra:

1. gradient variables w = (v1, v2, v3, T), T = p / rho;
2. lifting along each axis d: q_d = (2/h) [ D_d w + (1/w_N) delta_N (w* - w) - (1/w_0) delta_0 (w* - w) ]
   with the central value w* = (w_L + w_R)/2 at every face node;
3. viscous flux along d: (0, tau_1d, tau_2d, tau_3d, sum_k v_k tau_kd + kappa dT/dx_d) with
   tau = mu (grad v + grad v^T - (2/3) (div v) I), kappa = mu gamma / ((gamma - 1) Pr);
4. divergence: du/dt += (2/h) sum_d [ D_d f_v,d + lifting of (f* - f_v,d) ], f* the central
   flux in the face's normal direction.

At a hanging face the small side averages with the large side's values (of w, then of f_v)
interpolated to its nodes; the large side takes the L2 projection onto Q_N of the four quadrant
averages (the projection of ``dgsem3d.face_l2_projection``).  Every element's gradient comes from
the full stage state, so the partitioned RHS is again the mask of the full one.
"""

from __future__ import annotations

from collections import defaultdict

import numpy as np

from .dgsem3d import DGSEM3D, face_l2_projection
from .lgl import lagrange_basis


class NavierStokesDGSEM3D(DGSEM3D):
    def __init__(self, mesh, N: int = 2, surface_flux: str = "hlle", gamma: float = 1.4, mu: float = 1e-3,
                 prandtl: float = 0.72, chunk: int = 512):
        super().__init__(mesh, N, surface_flux, gamma, chunk)
        self.mu = mu
        self.kappa = mu * gamma / ((gamma - 1.0) * prandtl)

    def gradient_variables(self, V):
        rho = V[0]
        v = [V[1 + d] / rho for d in range(3)]
        p = (self.gamma - 1.0) * (V[4] - 0.5 * rho * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2))
        return np.stack([*v, p / rho])

    def _face_averages(self, W):
        """Central face values of the nodal field W [nv, e, k, j, i] on every element face:
        a list over faces of [nv, e, n, n] arrays."""
        nv, ne = W.shape[0], W.shape[1]
        n = self.N + 1
        out = [np.full((nv, ne, n, n), np.nan) for _ in range(6)]
        tr = [self.trace(W, f) for f in range(6)]
        for (A, B, d) in self.mesh.conforming:
            avg = 0.5 * (tr[2 * d + 1][:, A] + tr[2 * d][:, B])
            out[2 * d + 1][:, A] = avg
            out[2 * d][:, B] = avg
        quads = defaultdict(dict)
        for (A, B, d, large, q1, q2) in self.mesh.hanging:
            small, sface, lface = (B, 2 * d, 2 * d + 1) if large == A else (A, 2 * d + 1, 2 * d)
            s1 = 0.5 * (self.x + (2 * q1 - 1))
            s2 = 0.5 * (self.x + (2 * q2 - 1))
            li = np.einsum("pb,vba,qa->vpq", lagrange_basis(self.x, s2), tr[lface][:, large],
                           lagrange_basis(self.x, s1))
            avg = 0.5 * (tr[sface][:, small] + li)
            out[sface][:, small] = avg
            quads[(large, lface)][(q1, q2)] = avg
        for (large, lface), qv in quads.items():
            out[lface][:, large] = face_l2_projection(self.x, qv)
        return out

    def _strong_derivative(self, F, Fstar, d):
        """(2/h) [ D F + lifting of (F* - F) ] along axis d; F [nv, e, k, j, i]."""
        N = self.N
        w0, wN = self.w[0], self.w[N]
        if d == 0:
            G = np.einsum("im,vekjm->vekji", self.D, F)
        elif d == 1:
            G = np.einsum("jm,vekmi->vekji", self.D, F)
        else:
            G = np.einsum("km,vemji->vekji", self.D, F)
        lo = Fstar[2 * d] - self.trace(F, 2 * d)
        hi = Fstar[2 * d + 1] - self.trace(F, 2 * d + 1)
        if d == 0:
            G[..., 0] -= lo / w0
            G[..., N] += hi / wN
        elif d == 1:
            G[:, :, :, 0, :] -= lo / w0
            G[:, :, :, N, :] += hi / wN
        else:
            G[:, :, 0, :, :] -= lo / w0
            G[:, :, N, :, :] += hi / wN
        return (2.0 / self.mesh.h)[None, :, None, None, None] * G

    def gradients(self, V):
        W = self.gradient_variables(V)
        Ws = self._face_averages(W)
        return [self._strong_derivative(W, Ws, d) for d in range(3)]

    def viscous_fluxes(self, V, q):
        """f_v along each axis from the state and the gradients q[d] = d(v1, v2, v3, T)/dx_d."""
        rho = V[0]
        v = [V[1 + d] / rho for d in range(3)]
        mu, k = self.mu, self.kappa
        dv = [[q[b][a] for b in range(3)] for a in range(3)]          # dv[a][b] = d v_a / d x_b
        div = dv[0][0] + dv[1][1] + dv[2][2]
        tau = [[mu * (dv[a][b] + dv[b][a] - (2.0 / 3.0 if a == b else 0.0) * div) for b in range(3)]
               for a in range(3)]
        z = np.zeros_like(rho)
        out = []
        for d in range(3):
            energy = v[0] * tau[0][d] + v[1] * tau[1][d] + v[2] * tau[2][d] + k * q[d][3]
            out.append(np.stack([z, tau[0][d], tau[1][d], tau[2][d], energy]))
        return out

    def viscous_rhs(self, U: np.ndarray) -> np.ndarray:
        V = np.moveaxis(np.asarray(U, dtype=np.float64), 1, 0)
        q = self.gradients(V)
        f = self.viscous_fluxes(V, q)
        K = sum(self._strong_derivative(f[d], self._face_averages(f[d]), d) for d in range(3))
        return np.ascontiguousarray(np.moveaxis(K, 0, 1))

    def rhs(self, U: np.ndarray) -> np.ndarray:
        return super().rhs(U) + self.viscous_rhs(U)
