"""Adaptive refinement of the octree (oracle; test infrastructure only).

The paper's three-dimensional run (Sec. 7.1.3) refines the octree where the
enstrophy of Eq. Enstrophy, eps = rho |omega|^2 / 2 with the vorticity
omega = curl v, exceeds a threshold, from 16^3 cells up to two levels finer.
The oracle follows the 2D cycle (``amr.py``) with that indicator:

1. Indicator: eta_e = max over the element's nodes of rho |omega|^2 / 2, the
   velocity derivatives taken from the nodal polynomial, (2/h_e) D along each
   axis.
2. Desired level: level + 1 where eta > refine_above (up to level_max), level - 1
   where eta < coarsen_below (down to level_min), else level.
3. Constraints raised to their least fixed point: a cell coarsens only together
   with its seven siblings (all eight leaves, all wanting to coarsen); face
   neighbours differ by at most one level in the new mesh.
4. New leaves; transfer: a refined cell's children take the parent polynomial
   at their nodes (exact); a coarsened group's parent takes the L2 projection of
   the eight children's polynomials, computed from a 3D mass matrix and Gauss
   quadrature inside each child.
"""

from __future__ import annotations

from collections import defaultdict

import numpy as np
from numpy.polynomial import legendre as npleg

from perk_inputs.octree import morton_sort3

from .lgl import derivative_matrix, lagrange_basis, lgl_nodes_weights, mass_matrix_exact
from .octree import OctreeMesh


def enstrophy_indicator(U: np.ndarray, h: np.ndarray, N: int = 2) -> np.ndarray:
    """max over each element's nodes of rho |curl v|^2 / 2; U = [e, 5, k, j, i], h = [e]."""
    x, _ = lgl_nodes_weights(N)
    D = derivative_matrix(x)
    rho = U[:, 0]
    v = [U[:, 1 + d] / rho for d in range(3)]
    s = (2.0 / h)[:, None, None, None]

    def ddx(f):
        return s * np.einsum("im,ekjm->ekji", D, f)

    def ddy(f):
        return s * np.einsum("jm,ekmi->ekji", D, f)

    def ddz(f):
        return s * np.einsum("km,emji->ekji", D, f)

    wx = ddy(v[2]) - ddz(v[1])
    wy = ddz(v[0]) - ddx(v[2])
    wz = ddx(v[1]) - ddy(v[0])
    eps = 0.5 * rho * (wx * wx + wy * wy + wz * wz)
    return eps.reshape(len(U), -1).max(axis=1)


def desired_levels3(mesh: OctreeMesh, eta: np.ndarray, level_min: int, level_max: int, refine_above: float,
                    coarsen_below: float) -> np.ndarray:
    lev = mesh.cells[:, 0].astype(np.int64)
    d = lev.copy()
    d[(eta > refine_above) & (lev < level_max)] += 1
    d[(eta < coarsen_below) & (lev > level_min) & ~(eta > refine_above)] -= 1
    return balance3(mesh, d)


def balance3(mesh: OctreeMesh, d: np.ndarray) -> np.ndarray:
    """Least fixed point >= d of the sibling (eight leaves) and 2:1 face constraints."""
    lev = mesh.cells[:, 0].astype(np.int64)
    d = np.array(d, dtype=np.int64)
    groups = defaultdict(list)
    for e, (l, ix, iy, iz) in enumerate(mesh.cells.tolist()):
        if l > 0:
            groups[(l, ix // 2, iy // 2, iz // 2)].append(e)
    parent = [(int(l), int(ix) // 2, int(iy) // 2, int(iz) // 2) for (l, ix, iy, iz) in mesh.cells.tolist()]
    pairs = [(a, b) for (a, b, _) in mesh.conforming] + [(a, b) for (a, b, _, _, _, _) in mesh.hanging]
    changed = True
    while changed:
        changed = False
        for e in range(len(d)):
            if d[e] < lev[e]:
                g = groups[parent[e]] if lev[e] > 0 else []
                if len(g) != 8 or any(d[m] >= lev[m] or lev[m] != lev[e] for m in g):
                    for m in (g or [e]):
                        if d[m] < lev[m]:
                            d[m] = lev[m]
                            changed = True
        for (a, b) in pairs:
            if d[a] > d[b] + 1:
                d[b] = d[a] - 1
                changed = True
            elif d[b] > d[a] + 1:
                d[a] = d[b] - 1
                changed = True
    return d


def new_cells3(mesh: OctreeMesh, d: np.ndarray):
    out = set()
    for e, (l, ix, iy, iz) in enumerate(mesh.cells.tolist()):
        if d[e] == l + 1:
            for cz in (0, 1):
                for cy in (0, 1):
                    for cx in (0, 1):
                        out.add((l + 1, 2 * ix + cx, 2 * iy + cy, 2 * iz + cz))
        elif d[e] == l:
            out.add((l, ix, iy, iz))
        else:
            out.add((l - 1, ix // 2, iy // 2, iz // 2))
    return morton_sort3(out)


def transfer3(old_cells, U_old: np.ndarray, cells, N: int = 2) -> np.ndarray:
    """Solution on the new leaves: copy, interpolate (refine) or L2-project (coarsen)."""
    x, _ = lgl_nodes_weights(N)
    n = N + 1
    index = {tuple(int(v) for v in c): e for e, c in enumerate(old_cells)}
    xg, wg = npleg.leggauss(n + 1)
    M = mass_matrix_exact(x)
    M3 = np.kron(np.kron(M, M), M)                 # [(k,j,i),(c,b,a)] on the tensor basis
    Lc = lagrange_basis(x, xg)                     # child basis at the child's Gauss points
    W = np.einsum("r,q,p->rqp", wg, wg, wg) / 8.0  # child volume element in parent units
    U = np.zeros((len(cells), 5, n, n, n))
    for kk, (l, ix, iy, iz) in enumerate(cells):
        key = (l, ix, iy, iz)
        if key in index:
            U[kk] = U_old[index[key]]
            continue
        par = (l - 1, ix // 2, iy // 2, iz // 2)
        if par in index:
            Lx = lagrange_basis(x, 0.5 * (x + 2 * (ix % 2) - 1.0))
            Ly = lagrange_basis(x, 0.5 * (x + 2 * (iy % 2) - 1.0))
            Lz = lagrange_basis(x, 0.5 * (x + 2 * (iz % 2) - 1.0))
            U[kk] = np.einsum("kc,jb,ia,vcba->vkji", Lz, Ly, Lx, U_old[index[par]])
            continue
        rhs = np.zeros((5, n, n, n))
        for cz in (0, 1):
            for cy in (0, 1):
                for cx in (0, 1):
                    child = U_old[index[(l + 1, 2 * ix + cx, 2 * iy + cy, 2 * iz + cz)]]
                    f = np.einsum("rc,qb,pa,vcba->vrqp", Lc, Lc, Lc, child)   # values at (z, y, x) points
                    Px = lagrange_basis(x, 0.5 * (xg + 2 * cx - 1.0))
                    Py = lagrange_basis(x, 0.5 * (xg + 2 * cy - 1.0))
                    Pz = lagrange_basis(x, 0.5 * (xg + 2 * cz - 1.0))
                    rhs += np.einsum("vrqp,rqp,rk,qj,pi->vkji", f, W, Pz, Py, Px)
        U[kk] = np.linalg.solve(M3, rhs.reshape(5, -1).T).T.reshape(5, n, n, n)
    return U


def adapt3(mesh: OctreeMesh, U: np.ndarray, level_min: int, level_max: int, refine_above: float,
           coarsen_below: float, desired=None, N: int = 2):
    """One AMR cycle; returns (new OctreeMesh, transferred U, desired levels)."""
    if desired is None:
        desired = desired_levels3(mesh, enstrophy_indicator(U, mesh.h, N), level_min, level_max, refine_above,
                                  coarsen_below)
    cells = new_cells3(mesh, desired)
    U_new = transfer3([tuple(c) for c in mesh.cells.tolist()], U, cells, N)
    return OctreeMesh(np.asarray(cells), mesh.x0, mesh.length), U_new, desired
