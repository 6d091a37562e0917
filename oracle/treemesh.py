"""Face matching on a periodic quadtree leaf list (oracle; test infrastructure only).

The paper's TreeMesh (Sec. 6.2) couples leaf cells through faces of equal
size ("interfaces") and through 2:1 hanging faces ("mortars").  The oracle
finds every coupling by plain geometry: two cells touch when one's +x (or +y)
face and the other's -x (or -y) face lie on the same grid line (periodically)
and their extents overlap with positive length.  It never uses tree
connectivity, so it is independent of the library's tree walk.
"""

from __future__ import annotations

from collections import defaultdict
from dataclasses import dataclass, field

import numpy as np


@dataclass
class TreeMesh:
    cells: np.ndarray          # [n, 3] (level, ix, iy)
    x0: float
    length: float
    h: np.ndarray = field(init=False)          # physical cell size
    lo: np.ndarray = field(init=False)         # [n, 2] integer lower-left corner in finest units
    size: np.ndarray = field(init=False)       # extent in finest units
    lmax: int = field(init=False)

    def __post_init__(self):
        self.cells = np.asarray(self.cells, dtype=np.int64).reshape(-1, 3)
        lev = self.cells[:, 0]
        self.lmax = int(lev.max())
        self.size = (1 << (self.lmax - lev)).astype(np.int64)
        self.lo = np.stack([self.cells[:, 1] * self.size, self.cells[:, 2] * self.size], axis=1)
        self.h = self.length / (2.0 ** lev)
        self.conforming, self.hanging = match_faces(self.lo, self.size, 1 << self.lmax)

    @property
    def n_elem(self) -> int:
        return len(self.cells)


def match_faces(lo: np.ndarray, size: np.ndarray, D: int):
    """All face couplings of a periodic leaf list.

    Returns
      conforming: list of (A, B, d): the +d face of A meets the -d face of B, equal extent.
      hanging:    list of (A, B, d, large, half): A's +d face meets B's -d face with
                  unequal extents; ``large`` is A or B, ``half`` = 0 if the small
                  face covers the lower half of the large face, 1 for the upper half.
    """
    conforming = []
    hanging = []
    for d in (0, 1):
        t = 1 - d  # tangential axis
        minus_faces = defaultdict(list)
        for e in range(len(size)):
            minus_faces[int(lo[e, d])].append(e)
        for A in range(len(size)):
            line = int((lo[A, d] + size[A]) % D)
            a0 = int(lo[A, t])
            a1 = a0 + int(size[A])
            for B in minus_faces[line]:
                b0 = int(lo[B, t])
                b1 = b0 + int(size[B])
                if min(a1, b1) - max(a0, b0) <= 0:
                    continue
                if size[A] == size[B]:
                    conforming.append((A, B, d))
                elif size[A] > size[B]:
                    hanging.append((A, B, d, A, 0 if b0 == a0 else 1))
                else:
                    hanging.append((A, B, d, B, 0 if a0 == b0 else 1))
    return conforming, hanging


def is_balanced(mesh: TreeMesh) -> bool:
    """2:1 balance: every face coupling joins cells whose sizes differ by at most 2x,
    and every hanging face is split into exactly two halves."""
    for (A, B, d, large, half) in mesh.hanging:
        small = B if large == A else A
        if mesh.size[large] != 2 * mesh.size[small]:
            return False
    count = defaultdict(int)
    for (A, B, d, large, half) in mesh.hanging:
        count[(large, d, large == A)] += 1
    return all(v == 2 for v in count.values())
