"""DGSEM right-hand side on a periodic octree (oracle; test infrastructure only).

The three-dimensional counterpart of ``dgsem.py`` for the paper's Sec. 7.1.3
(the Taylor-Green vortex on an adaptively refined octree): the strong-form
DGSEM with flux differencing on hexahedral elements of size h with LGL nodes
x_i, weights w_i and derivative matrix D,

  du_ijk/dt = -(2/h) [ sum_m 2 D_im f#(u_ijk, u_mjk) + sum_m 2 D_jm g#(u_ijk, u_imk)
                       + sum_m 2 D_km h#(u_ijk, u_ijm) + surface terms ]

with, on each of the six faces, (1/w_N)(f* - f(u)) at the + face and
-(1/w_0)(f* - f(u)) at the - face (f* the numerical surface flux).  At a 2:1
hanging face (one large face, four small ones: the mortars of Kopriva 1996 on
faces) each small side takes the flux between its trace and the large side's
trace polynomial evaluated at its nodes; the large side takes the L2
projection onto Q_N of the piecewise polynomial formed by the four small-face
fluxes.  The projection here is computed from its definition on the square:
a Q_N mass matrix and right-hand side integrated by 2D Gauss quadrature (on
the whole face and on each quadrant), then one linear solve.

The partitioned right-hand side is the mask of the full one (Sec. 2.2).

Arrays are [n_elem, 5, n, n, n] indexed [e, var, k, j, i] with i along x,
j along y, k along z.
"""

from __future__ import annotations

from collections import defaultdict

import numpy as np
from numpy.polynomial import legendre as npleg

from . import euler3d
from .lgl import derivative_matrix, lagrange_basis, lgl_nodes_weights
from .octree import OctreeMesh

SURFACE_FLUXES = {"hll": euler3d.hll_flux, "hllc": euler3d.hllc_flux, "hlle": euler3d.hlle_flux,
                  "ec": euler3d.ec_flux}


def quad_basis(nodes: np.ndarray, s1: np.ndarray, s2: np.ndarray) -> np.ndarray:
    """Values of the Q_N Lagrange basis phi_(b, a)(s1, s2) = l_a(s1) l_b(s2) at the points
    (s1[p], s2[p]): array [points, n (b), n (a)]."""
    L1 = lagrange_basis(nodes, s1)      # [p, a]
    L2 = lagrange_basis(nodes, s2)      # [p, b]
    return L2[:, :, None] * L1[:, None, :]


def face_l2_projection(nodes: np.ndarray, quads) -> np.ndarray:
    """L2 projection onto Q_N on [-1, 1]^2 of the piecewise polynomial equal, on quadrant
    (q1, q2) = [q1 - 1, q1] x [q2 - 1, q2], to the interpolant of ``quads[(q1, q2)]``
    (values [..., n (t2), n (t1)] at the quadrant's own tensor nodes).  Returns [..., n, n]."""
    n = len(nodes)
    xg, wg = npleg.leggauss(n + 1)
    # every (Gauss point in t1, Gauss point in t2) pair of a square, as a flat point list
    g1, g2 = np.meshgrid(xg, xg, indexing="xy")
    w2d = np.outer(wg, wg).ravel()
    s1, s2 = g1.ravel(), g2.ravel()
    phi = quad_basis(nodes, s1, s2).reshape(len(s1), n * n)          # [p, (b, a)]
    M = phi.T @ (w2d[:, None] * phi)                                  # integral over the face
    rhs = 0.0
    for (q1, q2), f in quads.items():
        f = np.asarray(f)
        # physical face points of the quadrant (area 1/4 of the face) and their quadrant coordinates
        x1 = 0.5 * s1 + (q1 - 0.5)
        x2 = 0.5 * s2 + (q2 - 0.5)
        f_at = f.reshape(*f.shape[:-2], n * n) @ quad_basis(nodes, s1, s2).reshape(len(s1), n * n).T  # [..., p]
        phi_at = quad_basis(nodes, x1, x2).reshape(len(s1), n * n)
        rhs = rhs + (f_at * (0.25 * w2d)) @ phi_at
    rhs = np.asarray(rhs)
    sol = np.linalg.solve(M, rhs.reshape(-1, n * n).T).T
    return sol.reshape(*rhs.shape[:-1], n, n)


class DGSEM3D:
    def __init__(self, mesh: OctreeMesh, N: int = 2, surface_flux: str = "hlle", gamma: float = euler3d.GAMMA,
                 chunk: int = 512):
        self.mesh = mesh
        self.N = N
        self.gamma = gamma
        self.x, self.w = lgl_nodes_weights(N)
        self.D = derivative_matrix(self.x)
        self.fstar = SURFACE_FLUXES[surface_flux]
        self.chunk = chunk

    # ------------------------------------------------------------------ volume
    def _volume(self, V: np.ndarray) -> np.ndarray:
        """The three flux-differencing sums, V = [5, e, k, j, i]."""
        g = self.gamma
        twoD = 2.0 * self.D
        Fx = euler3d.ec_flux(V[..., :, None], V[..., None, :], 0, g)                          # [5,e,k,j,i,m]
        vol = np.einsum("im,vekjim->vekji", twoD, Fx)
        Fy = euler3d.ec_flux(V[:, :, :, :, None, :], V[:, :, :, None, :, :], 1, g)            # [5,e,k,j,m,i]
        vol += np.einsum("jm,vekjmi->vekji", twoD, Fy)
        Fz = euler3d.ec_flux(V[:, :, :, None, :, :], V[:, :, None, :, :, :], 2, g)            # [5,e,k,m,j,i]
        vol += np.einsum("km,vekmji->vekji", twoD, Fz)
        return vol

    # ----------------------------------------------------------------- surface
    def trace(self, V: np.ndarray, face: int) -> np.ndarray:
        """Face traces of every element [5, e, n (t2), n (t1)]; faces 0/1 = -x/+x, 2/3 = -y/+y,
        4/5 = -z/+z."""
        idx = 0 if face % 2 == 0 else self.N
        d = face // 2
        if d == 0:
            return V[:, :, :, :, idx]       # [5, e, k, j]: t2 = z, t1 = y
        if d == 1:
            return V[:, :, :, idx, :]       # [5, e, k, i]: t2 = z, t1 = x
        return V[:, :, idx, :, :]           # [5, e, j, i]: t2 = y, t1 = x

    def _face_fluxes(self, V: np.ndarray):
        """Numerical flux at the nodes of every element face: Fs[face] -> [5, e, n, n]."""
        g = self.gamma
        n = self.N + 1
        ne = V.shape[1]
        Fs = [np.full((5, ne, n, n), np.nan) for _ in range(6)]
        tr = [self.trace(V, f) for f in range(6)]
        conf = np.asarray(self.mesh.conforming, dtype=np.int64).reshape(-1, 3)
        for d in (0, 1, 2):
            sel = conf[conf[:, 2] == d]
            if len(sel) == 0:
                continue
            A, B = sel[:, 0], sel[:, 1]
            f = self.fstar(tr[2 * d + 1][:, A], tr[2 * d][:, B], d, g)
            Fs[2 * d + 1][:, A] = f
            Fs[2 * d][:, B] = f
        quads = defaultdict(dict)
        for (A, B, d, large, q1, q2) in self.mesh.hanging:
            if large == A:
                small, small_face, large_face = B, 2 * d, 2 * d + 1
            else:
                small, small_face, large_face = A, 2 * d + 1, 2 * d
            s1 = 0.5 * (self.x + (2 * q1 - 1))
            s2 = 0.5 * (self.x + (2 * q2 - 1))
            UL = tr[large_face][:, large]                                           # [5, b, a]
            u_large = np.einsum("pb,vba,qa->vpq", lagrange_basis(self.x, s2), UL, lagrange_basis(self.x, s1))
            u_small = tr[small_face][:, small]
            f = self.fstar(u_large, u_small, d, g) if large == A else self.fstar(u_small, u_large, d, g)
            Fs[small_face][:, small] = f
            quads[(large, large_face)][(q1, q2)] = f
        for (large, large_face), qv in quads.items():
            Fs[large_face][:, large] = face_l2_projection(self.x, qv)
        return Fs

    # --------------------------------------------------------------------- rhs
    def rhs(self, U: np.ndarray) -> np.ndarray:
        """Full DGSEM right-hand side F(U), shape [n_elem, 5, n, n, n]."""
        N = self.N
        g = self.gamma
        V = np.moveaxis(np.asarray(U, dtype=np.float64), 1, 0)            # [5, e, k, j, i]
        ne = V.shape[1]
        vol = np.empty_like(V)
        for s in range(0, ne, self.chunk):
            vol[:, s:s + self.chunk] = self._volume(V[:, s:s + self.chunk])
        Fs = self._face_fluxes(V)
        Sf = np.zeros_like(V)
        w0, wN = self.w[0], self.w[N]
        for face in range(6):
            d = face // 2
            jump = Fs[face] - euler3d.physical_flux(self.trace(V, face), d, g)
            idx = 0 if face % 2 == 0 else N
            sign = -1.0 / w0 if face % 2 == 0 else 1.0 / wN
            if d == 0:
                Sf[:, :, :, :, idx] += sign * jump
            elif d == 1:
                Sf[:, :, :, idx, :] += sign * jump
            else:
                Sf[:, :, idx, :, :] += sign * jump
        h = self.mesh.h
        K = -(2.0 / h)[None, :, None, None, None] * (vol + Sf)
        return np.ascontiguousarray(np.moveaxis(K, 0, 1))

    def rhs_masked(self, U: np.ndarray, active: np.ndarray) -> np.ndarray:
        """I^(active) F(U): the full RHS with inactive elements set to zero."""
        return self.rhs(U) * np.asarray(active, dtype=np.float64)[:, None, None, None, None]

    # -------------------------------------------------------------- utilities
    def integrate(self, U: np.ndarray) -> np.ndarray:
        """Domain integral of each conserved variable: sum_e (h_e/2)^3 sum_ijk w_i w_j w_k u."""
        W = np.einsum("k,j,i->kji", self.w, self.w, self.w)
        return np.einsum("e,evkji,kji->v", (0.5 * self.mesh.h) ** 3, U, W)


def max_wave_speed_dt3(U: np.ndarray, h: np.ndarray, N: int, cfl: float, gamma: float = euler3d.GAMMA) -> float:
    """dt = cfl * min_e h_e / ((N + 1) lambda_e), lambda_e = max over the element's nodes of
    |v1| + |v2| + |v3| + 3c (the 2D rule of Eq. TimestepConstraint summed over three axes).
    NaN if any node has rho <= 0, p <= 0 or a non-finite entry (no sound speed exists)."""
    rho = U[:, 0]
    with np.errstate(divide="ignore", invalid="ignore"):
        v = [U[:, 1 + d] / rho for d in range(3)]
        p = (gamma - 1.0) * (U[:, 4] - 0.5 * rho * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2))
        if not (np.all(rho > 0.0) and np.all(p > 0.0)):
            return float("nan")
        c = np.sqrt(gamma * p / rho)
    lam = (np.abs(v[0]) + np.abs(v[1]) + np.abs(v[2]) + 3.0 * c).reshape(len(h), -1).max(axis=1)
    return float(cfl * np.min(h / ((N + 1) * lam)))
