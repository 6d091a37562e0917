"""Adaptive mesh refinement of the quadtree (oracle; test infrastructure only).

The paper adapts the TreeMesh every N_AMR steps (Sec. 7; the AMR callback
before the partition is re-assigned, Sec. 6.2).  The oracle follows these steps:

1. Indicator, one of
   - density gradient: eta_e = h_e max_nodes |grad rho| / mean_e(rho), with
     grad rho = (2/h_e) (D rho along x, D rho along y) at the nodes and the mean
     by the LGL quadrature; eta is dimensionless;
   - Loehner's second-difference estimator (Loehner 1987, in the nodal form of
     the FLASH code, Fryxell et al. 2000) of the velocity v_x, the indicator of
     the shear-layer run (Sec. 7.1.1): for every three consecutive nodes
     u_-, u_0, u_+ along a grid line of the element, in both directions,
       |u_+ - 2 u_0 + u_-| / (|u_+ - u_0| + |u_0 - u_-| + eps (|u_+| + 2|u_0| + |u_-|)),
     eta_e = the largest of these (0 where the denominator vanishes), eps = 0.2.
2. Desired level: level + 1 where eta > refine_above (up to level_max),
   level - 1 where eta < coarsen_below (down to level_min), else level.
3. Constraints, raised to their least fixed point: a cell may only coarsen
   together with its three siblings (all four leaves, all wanting to coarsen);
   face neighbours may differ by at most one level in the new mesh.
4. New leaves; solution transfer: a refined cell's children take the parent
   polynomial evaluated at their nodes (exact); a coarsened group's parent takes
   the L2 projection of the four children's polynomials.
"""

from __future__ import annotations

from collections import defaultdict

import numpy as np
from numpy.polynomial import legendre as npleg

from perk_inputs import morton_sort

from .lgl import derivative_matrix, lagrange_basis, lgl_nodes_weights, mass_matrix_exact
from .treemesh import TreeMesh


LOHNER_EPS = 0.2


def lohner_indicator(f: np.ndarray, eps: float = LOHNER_EPS) -> np.ndarray:
    """Loehner's estimator of the nodal field f [e, j, i] (largest over the node triples)."""
    out = np.zeros(len(f))
    for line_major in (False, True):
        g = np.swapaxes(f, 1, 2) if line_major else f        # triples along i (x), then along j (y)
        for c in range(1, g.shape[2] - 1):
            um, u0, up = g[:, :, c - 1], g[:, :, c], g[:, :, c + 1]
            num = np.abs(up - 2.0 * u0 + um)
            den = np.abs(up - u0) + np.abs(u0 - um) + eps * (np.abs(up) + 2.0 * np.abs(u0) + np.abs(um))
            r = np.where(den > 0.0, num / np.where(den > 0.0, den, 1.0), 0.0)
            out = np.maximum(out, r.max(axis=1))
    return out


def indicator(U: np.ndarray, N: int = 3, kind: str = "density") -> np.ndarray:
    if kind == "lohner_vx":
        return lohner_indicator(U[:, 1] / U[:, 0])
    if kind != "density":
        raise ValueError(kind)
    x, w = lgl_nodes_weights(N)
    D = derivative_matrix(x)
    rho = U[:, 0]                                              # [e, j, i]
    gx = np.einsum("im,ejm->eji", D, rho)                      # d rho / d xi (reference), x
    gy = np.einsum("jm,emi->eji", D, rho)                      # y
    mean = np.einsum("ji,eji->e", np.outer(w, w), rho) / 4.0
    # h |grad rho| = h (2/h) |grad_xi rho|
    return 2.0 * np.sqrt(gx * gx + gy * gy).reshape(len(rho), -1).max(axis=1) / mean


def desired_levels(mesh: TreeMesh, eta: np.ndarray, level_min: int, level_max: int, refine_above: float,
                   coarsen_below: float) -> np.ndarray:
    lev = mesh.cells[:, 0].astype(np.int64)
    d = lev.copy()
    d[(eta > refine_above) & (lev < level_max)] += 1
    d[(eta < coarsen_below) & (lev > level_min) & ~(eta > refine_above)] -= 1
    return balance(mesh, d)


def balance(mesh: TreeMesh, d: np.ndarray) -> np.ndarray:
    """Least fixed point >= d of the sibling and 2:1 face constraints."""
    lev = mesh.cells[:, 0].astype(np.int64)
    d = np.array(d, dtype=np.int64)
    groups = defaultdict(list)
    for e, (l, ix, iy) in enumerate(mesh.cells):
        if l > 0:
            groups[(int(l), int(ix) // 2, int(iy) // 2)].append(e)
    pairs = [(a, b) for (a, b, _) in mesh.conforming] + [(a, b) for (a, b, _, _, _) in mesh.hanging]
    changed = True
    while changed:
        changed = False
        for e in range(len(d)):
            if d[e] < lev[e]:
                g = groups[(int(lev[e]), int(mesh.cells[e, 1]) // 2, int(mesh.cells[e, 2]) // 2)]
                if len(g) != 4 or any(d[m] >= lev[m] or lev[m] != lev[e] for m in g):
                    for m in g:
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


def new_cells(mesh: TreeMesh, d: np.ndarray):
    out = set()
    for e, (l, ix, iy) in enumerate(mesh.cells):
        l, ix, iy = int(l), int(ix), int(iy)
        if d[e] == l + 1:
            for cy in (0, 1):
                for cx in (0, 1):
                    out.add((l + 1, 2 * ix + cx, 2 * iy + cy))
        elif d[e] == l:
            out.add((l, ix, iy))
        else:
            out.add((l - 1, ix // 2, iy // 2))
    return morton_sort(out)


def transfer(old_cells, U_old: np.ndarray, cells, N: int = 3) -> np.ndarray:
    """Solution on the new leaves: copy, interpolate (refine) or L2-project (coarsen)."""
    x, w = lgl_nodes_weights(N)
    n = N + 1
    index = {tuple(int(v) for v in c): e for e, c in enumerate(old_cells)}
    xg, wg = npleg.leggauss(n + 1)
    M = mass_matrix_exact(x)
    M2 = np.kron(M, M)                                         # [(j,i),(b,a)] on the tensor basis
    U = np.zeros((len(cells), 4, n, n))
    for k, (l, ix, iy) in enumerate(cells):
        key = (l, ix, iy)
        if key in index:
            U[k] = U_old[index[key]]
            continue
        parent = (l - 1, ix // 2, iy // 2)
        if parent in index:
            cx, cy = ix % 2, iy % 2
            Lx = lagrange_basis(x, 0.5 * (x + 2 * cx - 1.0))   # [i, a]
            Ly = lagrange_basis(x, 0.5 * (x + 2 * cy - 1.0))   # [j, b]
            U[k] = np.einsum("jb,ia,vba->vji", Ly, Lx, U_old[index[parent]])
            continue
        # coarsening: L2 projection of the four children (Gauss quadrature inside each child)
        rhs = np.zeros((4, n, n))
        for cy in (0, 1):
            for cx in (0, 1):
                child = U_old[index[(l + 1, 2 * ix + cx, 2 * iy + cy)]]
                # child quadrature points in child reference coordinates and in parent coordinates
                Lc = lagrange_basis(x, xg)                    # child basis at child Gauss points
                px = 0.5 * (xg + 2 * cx - 1.0)
                py = 0.5 * (xg + 2 * cy - 1.0)
                Pbx = lagrange_basis(x, px)                   # parent basis at those points
                Pby = lagrange_basis(x, py)
                f = np.einsum("qb,pa,vba->vqp", Lc, Lc, child)        # child values at (q: y, p: x)
                W = 0.25 * np.outer(wg, wg)                            # dA of the child, in parent units
                rhs += np.einsum("vqp,qp,qj,pi->vji", f, W, Pby, Pbx)
        U[k] = np.linalg.solve(M2, rhs.reshape(4, -1).T).T.reshape(4, n, n)
    return U


def adapt(mesh: TreeMesh, U: np.ndarray, level_min: int, level_max: int, refine_above: float, coarsen_below: float,
          desired=None, kind: str = "density"):
    """One AMR cycle; returns (new TreeMesh, transferred U, desired levels)."""
    if desired is None:
        desired = desired_levels(mesh, indicator(U, kind=kind), level_min, level_max, refine_above, coarsen_below)
    cells = new_cells(mesh, desired)
    U_new = transfer([tuple(c) for c in mesh.cells.tolist()], U, cells)
    return TreeMesh(cells, mesh.x0, mesh.length), U_new, desired
