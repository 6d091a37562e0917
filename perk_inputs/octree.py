"""Octree leaf-cell lists and 3D initial states for the three-dimensional workload.

A cell is ``(level, ix, iy, iz)``: level 0 is the whole cube and a cell of level
``l`` covers ``[ix, ix+1) x [iy, iy+1) x [iz, iz+1)`` in units of ``L / 2**l``.
Lists are returned in Morton order of the cells' lower corners (the depth-first
leaf order of an octree).  Initial states are sampled at tensor-product nodes
whose 1D reference positions the caller supplies.  Nothing here discretises
anything.
"""

from __future__ import annotations

import math
from typing import Callable, Iterable, List, Sequence, Tuple

import numpy as np

from .initial import GAMMA, SEED

Cell3 = Tuple[int, int, int, int]


def _interleave3(x: int, y: int, z: int) -> int:
    m = 0
    for b in range(21):
        m |= ((x >> b) & 1) << (3 * b)
        m |= ((y >> b) & 1) << (3 * b + 1)
        m |= ((z >> b) & 1) << (3 * b + 2)
    return m


def morton_sort3(cells: Iterable[Cell3]) -> List[Cell3]:
    cells = list(cells)
    lmax = max(c[0] for c in cells)
    return sorted(cells, key=lambda c: (_interleave3(c[1] << (lmax - c[0]), c[2] << (lmax - c[0]),
                                                     c[3] << (lmax - c[0])), c[0]))


def uniform_cells3(level: int) -> List[Cell3]:
    n = 1 << level
    return morton_sort3([(level, ix, iy, iz) for iz in range(n) for iy in range(n) for ix in range(n)])


def refine_cells3(cells: Iterable[Cell3], pred: Callable[[int, int, int, int], bool]) -> List[Cell3]:
    """Replace every cell for which ``pred(level, ix, iy, iz)`` holds by its eight children."""
    out: List[Cell3] = []
    for (l, ix, iy, iz) in cells:
        if pred(l, ix, iy, iz):
            for cz in (0, 1):
                for cy in (0, 1):
                    for cx in (0, 1):
                        out.append((l + 1, 2 * ix + cx, 2 * iy + cy, 2 * iz + cz))
        else:
            out.append((l, ix, iy, iz))
    return morton_sort3(out)


def block_refined_cells3(base_level: int = 2, lo: int = 1, hi: int = 3) -> List[Cell3]:
    """Uniform base mesh with the block of base cells ``lo <= ix, iy, iz < hi`` refined once
    (``2, 1, 3``: 56 coarse and 64 fine cells, a two-level mesh with hanging faces on
    every side of the block)."""
    return refine_cells3(uniform_cells3(base_level),
                         lambda l, ix, iy, iz: lo <= ix < hi and lo <= iy < hi and lo <= iz < hi)


def slab_cells3(level_min: int = 4, level_max: int = 6, width: float = 1.0 / 32.0) -> List[Cell3]:
    """Graded mesh refined towards the plane z = L/2: within ``width`` (in domain units)
    of the plane the target level is ``level_max``; each further band of the next
    coarser level is two of its own cells thick, so face neighbours differ by at most
    one level.  ``4, 6, 1/32``: a level-6 slab four cells thick (16,384 cells), level-5 bands
    three cells thick on either side (6,144) and a level-4 background (3,072): 25,600 cells."""

    def target(l: int, iz: int) -> int:
        zc = (iz + 0.5) / (1 << l)
        d = abs(zc - 0.5)
        lev = level_max
        w = width
        while lev > level_min and d > w:
            lev -= 1
            w = w + 2.0 / (1 << lev)
        return lev

    cells = uniform_cells3(level_min)
    for _ in range(level_max - level_min):
        cells = refine_cells3(cells, lambda l, ix, iy, iz: target(l, iz) > l)
    return cells


def extrude_cells(cells2d: Sequence[Tuple[int, int, int]]) -> List[Cell3]:
    """The octree whose cells are the quadtree cells of ``cells2d`` repeated along z at
    their own level (every column of a 2D cell of level l holds 2**l cubes)."""
    out = []
    for (l, ix, iy) in cells2d:
        for iz in range(1 << l):
            out.append((l, ix, iy, iz))
    return morton_sort3(out)


def prim_to_cons3(rho, v1, v2, v3, p, gamma: float = GAMMA):
    return np.stack([rho, rho * v1, rho * v2, rho * v3,
                     p / (gamma - 1.0) + 0.5 * rho * (v1 * v1 + v2 * v2 + v3 * v3)])


def taylor_green(x, y, z, *, mach: float = 0.1, gamma: float = GAMMA):
    """Taylor-Green vortex on [0, 2 pi]^3 (the paper's Eq. IC_TaylorGreen): unit density,
    v = (sin x cos y cos z, -cos x sin y cos z, 0), p = p0 + ((cos 2x + cos 2y)(2 + cos 2z)) / 16
    with p0 = 1 / (mach^2 gamma)."""
    rho = np.ones_like(x)
    v1 = np.sin(x) * np.cos(y) * np.cos(z)
    v2 = -np.cos(x) * np.sin(y) * np.cos(z)
    v3 = np.zeros_like(x)
    p0 = 1.0 / (mach * mach * gamma)
    p = p0 + (np.cos(2.0 * x) + np.cos(2.0 * y)) * (2.0 + np.cos(2.0 * z)) / 16.0
    return prim_to_cons3(rho, v1, v2, v3, p, gamma)


def density_wave3(x, y, z, t: float = 0.0, *, period: float = 2.0, velocity=(0.3, -0.2, 0.5),
                  amplitude: float = 0.2, pressure: float = 1.0, gamma: float = GAMMA):
    """Exact solution of the Euler equations: a density wave
    rho = 1 + amplitude sin(2 pi (x + y + z - (v1 + v2 + v3) t) / period) carried by a
    constant velocity at constant pressure."""
    v1, v2, v3 = velocity
    phase = 2.0 * math.pi * ((x - v1 * t) + (y - v2 * t) + (z - v3 * t)) / period
    rho = 1.0 + amplitude * np.sin(phase)
    one = np.ones_like(rho)
    return prim_to_cons3(rho, v1 * one, v2 * one, v3 * one, pressure * one, gamma)


def node_coordinates3(cells: Sequence, x0: float, length: float, xi: np.ndarray):
    """Physical coordinates ``(X, Y, Z)`` of the tensor-product nodes of every cell, each of
    shape ``[n_cells, n, n, n]`` indexed ``[e, k, j, i]`` (i along x, j along y, k along z)."""
    cells = np.asarray(cells, dtype=np.int64).reshape(-1, 4)
    lev = cells[:, 0]
    h = length / (2.0 ** lev)
    s = 0.5 * (np.asarray(xi, dtype=np.float64) + 1.0)
    n = len(s)
    lo = [x0 + cells[:, 1 + d] * h for d in range(3)]
    X = lo[0][:, None, None, None] + h[:, None, None, None] * s[None, None, None, :]
    Y = lo[1][:, None, None, None] + h[:, None, None, None] * s[None, None, :, None]
    Z = lo[2][:, None, None, None] + h[:, None, None, None] * s[None, :, None, None]
    shape = (len(cells), n, n, n)
    return (np.broadcast_to(X, shape).copy(), np.broadcast_to(Y, shape).copy(), np.broadcast_to(Z, shape).copy())


def nodal_state3(ic, cells: Sequence, x0: float, length: float, xi: np.ndarray, **kw) -> np.ndarray:
    """Initial condition ``ic(x, y, z)`` sampled at the nodes: array ``[n_cells, 5, n, n, n]``,
    C-contiguous float64."""
    X, Y, Z = node_coordinates3(cells, x0, length, xi)
    U = ic(X, Y, Z, **kw)
    return np.ascontiguousarray(np.moveaxis(U, 0, 1), dtype=np.float64)


def smooth_random_state3(cells: Sequence, x0: float, length: float, xi: np.ndarray, seed: int = SEED + 300,
                         n_modes: int = 3, amplitude: float = 0.05) -> np.ndarray:
    """Seeded smooth, positive 3D state: background (rho, v1, v2, v3, p) = (1, 0.3, -0.2, 0.1, 1)
    plus a few random periodic Fourier modes of each primitive variable."""
    rng = np.random.default_rng(seed)
    X, Y, Z = node_coordinates3(cells, x0, length, xi)
    k = 2.0 * math.pi / length
    prims = []
    for base in (1.0, 0.3, -0.2, 0.1, 1.0):
        f = np.full_like(X, base)
        for _ in range(n_modes):
            a = amplitude * rng.uniform(-1.0, 1.0)
            mx, my, mz = rng.integers(0, 3, size=3)
            ph = rng.uniform(0.0, 2.0 * math.pi)
            f = f + a * np.sin(k * (mx * (X - x0) + my * (Y - x0) + mz * (Z - x0)) + ph)
        prims.append(f)
    U = prim_to_cons3(*prims)
    return np.ascontiguousarray(np.moveaxis(U, 0, 1), dtype=np.float64)
