"""DGSEM right-hand side on a periodic quadtree (oracle; test infrastructure only).

F(U) is the standard strong-form DGSEM with flux differencing (the spatial
discretisation of the paper's Sec. 6.1; Gassner 2013/2016 split forms): on an
element of size h with LGL nodes x_i, weights w_i and derivative matrix D,

  du_ij/dt = -(2/h) [ sum_m 2 D_im f#(u_ij, u_mj) + sum_m 2 D_jm g#(u_ij, u_im)
                      + (1/w_N) delta_iN (f*_+x,j - f(u_Nj)) - (1/w_0) delta_i0 (f*_-x,j - f(u_0j))
                      + (1/w_N) delta_jN (g*_+y,i - g(u_iN)) - (1/w_0) delta_j0 (g*_-y,i - g(u_i0)) ]

with f#, g# the two-point volume flux in x and y (the m = i term is the
physical flux, since f#(u, u) = f(u)) and f*, g* the numerical surface flux.
At a 2:1 hanging face (mortar, Kopriva 1996) the small side takes the flux
between its trace and the large side's trace polynomial evaluated at its
nodes; the large side takes the L2 projection of the two half-face fluxes.

The partitioned right-hand side of stage i is the mask of the full one
(Sec. 2.2): F^(r)(U) = I^(r) F(U); the oracle always evaluates F on every
element and masks afterwards.

Arrays are [n_elem, 4, n, n] indexed [e, var, j, i] with i along x.
"""

from __future__ import annotations

from collections import defaultdict

import numpy as np

from . import euler
from .lgl import derivative_matrix, lagrange_eval, l2_project_two_halves, lgl_nodes_weights
from .treemesh import TreeMesh

SURFACE_FLUXES = {"hll": euler.hll_flux, "hllc": euler.hllc_flux, "ec": euler.ec_flux, "hlle": euler.hlle_flux}


class DGSEM:
    def __init__(self, mesh: TreeMesh, N: int = 3, surface_flux: str = "hll", gamma: float = euler.GAMMA,
                 chunk: int = 4096):
        self.mesh = mesh
        self.N = N
        self.gamma = gamma
        self.x, self.w = lgl_nodes_weights(N)
        self.D = derivative_matrix(self.x)
        self.fstar = SURFACE_FLUXES[surface_flux]
        self.chunk = chunk

    # ------------------------------------------------------------------ volume
    def _volume(self, V: np.ndarray) -> np.ndarray:
        """sum_m 2 D_im f#(u_ij, u_mj) + sum_m 2 D_jm g#(u_ij, u_im), V = [4, e, j, i]."""
        g = self.gamma
        twoD = 2.0 * self.D
        Fx = euler.ec_flux(V[:, :, :, :, None], V[:, :, :, None, :], 0, g)    # [4, e, j, i, m]
        vol = np.einsum("im,vejim->veji", twoD, Fx)
        Fy = euler.ec_flux(V[:, :, :, None, :], V[:, :, None, :, :], 1, g)    # [4, e, j, m, i]
        vol += np.einsum("jm,vejmi->veji", twoD, Fy)
        return vol

    # ----------------------------------------------------------------- surface
    def _face_fluxes(self, V: np.ndarray):
        """Numerical flux at the nodes of every element face: Fs[e][face] -> [4, n].
        Faces: 0 = -x (i = 0), 1 = +x (i = N), 2 = -y (j = 0), 3 = +y (j = N)."""
        N = self.N
        g = self.gamma

        def trace(e, face):
            if face == 0:
                return V[:, e, :, 0]
            if face == 1:
                return V[:, e, :, N]
            if face == 2:
                return V[:, e, 0, :]
            return V[:, e, N, :]

        Fs = {}
        conf = self.mesh.conforming
        if conf:
            A = np.array([c[0] for c in conf])
            B = np.array([c[1] for c in conf])
            d = np.array([c[2] for c in conf])
            for dd in (0, 1):
                sel = d == dd
                if not np.any(sel):
                    continue
                uA = np.stack([trace(a, 2 * dd + 1) for a in A[sel]], axis=1)   # [4, k, n]
                uB = np.stack([trace(b, 2 * dd) for b in B[sel]], axis=1)
                f = self.fstar(uA, uB, dd, g)
                for k, (a, b) in enumerate(zip(A[sel], B[sel])):
                    Fs[(int(a), 2 * dd + 1)] = f[:, k]
                    Fs[(int(b), 2 * dd)] = f[:, k]
        halves = defaultdict(dict)
        for (Ae, Be, d, large, half) in self.mesh.hanging:
            if large == Ae:
                small, small_face, large_face = Be, 2 * d, 2 * d + 1
            else:
                small, small_face, large_face = Ae, 2 * d + 1, 2 * d
            s = 0.5 * (self.x - 1.0) if half == 0 else 0.5 * (self.x + 1.0)
            u_large = lagrange_eval(self.x, trace(large, large_face), s)          # [4, n]
            u_small = trace(small, small_face)
            f = self.fstar(u_large, u_small, d, g) if large == Ae else self.fstar(u_small, u_large, d, g)
            Fs[(int(small), small_face)] = f
            halves[(int(large), large_face)][half] = f
        for key, hv in halves.items():
            Fs[key] = l2_project_two_halves(self.x, hv[0], hv[1])
        return Fs

    # --------------------------------------------------------------------- rhs
    def rhs(self, U: np.ndarray) -> np.ndarray:
        """Full DGSEM right-hand side F(U), shape [n_elem, 4, n, n]."""
        N = self.N
        g = self.gamma
        V = np.moveaxis(np.asarray(U, dtype=np.float64), 1, 0)            # [4, e, j, i]
        ne = V.shape[1]
        vol = np.empty_like(V)
        for s in range(0, ne, self.chunk):
            vol[:, s:s + self.chunk] = self._volume(V[:, s:s + self.chunk])
        Fs = self._face_fluxes(V)
        S = np.zeros_like(V)
        w0, wN = self.w[0], self.w[N]
        for e in range(ne):
            fx0 = euler.physical_flux(V[:, e, :, 0], 0, g)
            fxN = euler.physical_flux(V[:, e, :, N], 0, g)
            fy0 = euler.physical_flux(V[:, e, 0, :], 1, g)
            fyN = euler.physical_flux(V[:, e, N, :], 1, g)
            S[:, e, :, 0] -= (Fs[(e, 0)] - fx0) / w0
            S[:, e, :, N] += (Fs[(e, 1)] - fxN) / wN
            S[:, e, 0, :] -= (Fs[(e, 2)] - fy0) / w0
            S[:, e, N, :] += (Fs[(e, 3)] - fyN) / wN
        h = self.mesh.h
        K = -(2.0 / h)[None, :, None, None] * (vol + S)
        return np.ascontiguousarray(np.moveaxis(K, 0, 1))

    def rhs_masked(self, U: np.ndarray, active: np.ndarray) -> np.ndarray:
        """I^(active) F(U): the full RHS with inactive elements set to zero."""
        return self.rhs(U) * np.asarray(active, dtype=np.float64)[:, None, None, None]

    # -------------------------------------------------------------- utilities
    def integrate(self, U: np.ndarray) -> np.ndarray:
        """Domain integral of each conserved variable: sum_e (h_e/2)^2 sum_ij w_i w_j u."""
        W = np.outer(self.w, self.w)
        return np.einsum("e,evji,ji->v", (0.5 * self.mesh.h) ** 2, U, W)
