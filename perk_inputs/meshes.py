"""Quadtree leaf-cell lists for the synthetic workloads.

A cell is ``(level, ix, iy)``: level 0 is the whole square domain and a cell of
level ``l`` covers ``[ix, ix+1) x [iy, iy+1)`` in units of ``L / 2**l``.  A
mesh is the list of its leaf cells; list order is element order (the row of
the solution array that belongs to the cell).  Lists are returned in Morton
(Z-curve) order of the cells' lower-left corners, which is the depth-first
leaf order of a quadtree.
"""

from __future__ import annotations

from typing import Callable, Iterable, List, Tuple

Cell = Tuple[int, int, int]


def uniform_cells(level: int) -> List[Cell]:
    n = 1 << level
    return morton_sort([(level, ix, iy) for iy in range(n) for ix in range(n)])


def refine_cells(cells: Iterable[Cell], pred: Callable[[int, int, int], bool]) -> List[Cell]:
    """Replace every cell for which ``pred(level, ix, iy)`` holds by its four children."""
    out: List[Cell] = []
    for (l, ix, iy) in cells:
        if pred(l, ix, iy):
            for cy in (0, 1):
                for cx in (0, 1):
                    out.append((l + 1, 2 * ix + cx, 2 * iy + cy))
        else:
            out.append((l, ix, iy))
    return morton_sort(out)


def _interleave(x: int, y: int) -> int:
    z = 0
    for b in range(32):
        z |= ((x >> b) & 1) << (2 * b)
        z |= ((y >> b) & 1) << (2 * b + 1)
    return z


def morton_sort(cells: Iterable[Cell]) -> List[Cell]:
    cells = list(cells)
    lmax = max(c[0] for c in cells)
    return sorted(cells, key=lambda c: (_interleave(c[1] << (lmax - c[0]), c[2] << (lmax - c[0])), c[0]))


def vortex_two_level_cells(base_level: int = 4, lo: int = 4, hi: int = 12) -> List[Cell]:
    """Uniform base mesh with the block of base cells ``lo <= ix, iy < hi`` refined once.

    ``base_level=4, lo=4, hi=12`` is the 16x16 vortex mesh with its central
    8x8 block refined (448 cells, 32 hanging faces); ``base_level=8, lo=64,
    hi=192`` is the 256x256 variant with the central 128x128 block refined.
    """
    return refine_cells(uniform_cells(base_level),
                        lambda l, ix, iy: lo <= ix < hi and lo <= iy < hi)


def _graded_band_levels(level_min: int, level_max: int, centers, width: float):
    """Target level of a cell from the distance of its centre to the nearest
    horizontal line ``y = c`` (coordinates in units of the domain, [0, 1)).

    Within ``width`` of a line the target is ``level_max``; each further band
    of the next coarser level is two of its own cells wide.
    """

    def target(l: int, ix: int, iy: int) -> int:
        yc = (iy + 0.5) / (1 << l)
        d = min(min(abs(yc - c), 1.0 - abs(yc - c)) for c in centers)
        lev = level_max
        w = width
        while lev > level_min and d > w:
            lev -= 1
            w = w + 2.0 / (1 << lev)
        return lev

    return target


def kh_band_cells(level_min: int = 4, level_max: int = 7, width: float = 0.06) -> List[Cell]:
    """Static graded mesh refined towards the two shear lines of the
    Kelvin-Helmholtz initial state (y = -0.5 and y = +0.5 on [-1, 1]^2, i.e.
    0.25 and 0.75 in domain units)."""
    target = _graded_band_levels(level_min, level_max, (0.25, 0.75), width)
    cells = uniform_cells(level_min)
    for _ in range(level_max - level_min):
        cells = refine_cells(cells, lambda l, ix, iy: target(l, ix, iy) > l)
    return cells


def nested_band_cells(level_min: int = 2, level_max: int = 5, center: float = 0.75) -> List[Cell]:
    """Mesh refined towards one horizontal line ``y = center`` (domain units, [0, 1)): at every
    level the cells whose centres lie within 1.5 of their own widths of the line are refined,
    so each level forms a band two cells high around the next finer one (2:1 balanced).  With
    the defaults: four levels 2..5, 184 cells, the upper shear line of the Kelvin-Helmholtz
    state on [-1, 1]^2."""
    cells = uniform_cells(level_min)
    for _ in range(level_max - level_min):
        def near(l: int, ix: int, iy: int) -> bool:
            d = abs((iy + 0.5) / (1 << l) - center)
            return min(d, 1.0 - d) < 1.5 / (1 << l)
        cells = refine_cells(cells, near)
    return cells


def three_level_band_cells(level_min: int = 5, level_max: int = 7, width: float = 0.1) -> List[Cell]:
    """Frozen three-level graded mesh around the shear lines (adjoint window)."""
    return kh_band_cells(level_min, level_max, width)
