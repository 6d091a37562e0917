"""Face matching on a periodic octree leaf list (oracle; test infrastructure only).

The three-dimensional run of the paper (Sec. 7.1.3) uses the TreeMesh of
Sec. 6.2 in 3D: cubic leaf cells of an octree, coupled through faces of equal
size ("interfaces") and through 2:1 hanging faces, where one large face meets
four small ones ("mortars").  As in the 2D oracle, every coupling is found by
plain geometry (two cells touch when one's +d face and the other's -d face lie
in the same plane, periodically, and the two squares overlap with positive
area); tree connectivity is never used.

Face node order: the face normal to axis d has the two other axes t1 < t2 as
its tangential axes; a face trace is an array [var, n (along t2), n (along t1)].
"""

from __future__ import annotations

from collections import defaultdict
from dataclasses import dataclass, field

import numpy as np

TANGENTIAL = {0: (1, 2), 1: (0, 2), 2: (0, 1)}


@dataclass
class OctreeMesh:
    cells: np.ndarray          # [n, 4] (level, ix, iy, iz)
    x0: float
    length: float
    h: np.ndarray = field(init=False)          # physical cell size
    lo: np.ndarray = field(init=False)         # [n, 3] integer lower corner in finest units
    size: np.ndarray = field(init=False)       # extent in finest units
    lmax: int = field(init=False)

    def __post_init__(self):
        self.cells = np.asarray(self.cells, dtype=np.int64).reshape(-1, 4)
        lev = self.cells[:, 0]
        self.lmax = int(lev.max())
        self.size = (1 << (self.lmax - lev)).astype(np.int64)
        self.lo = self.cells[:, 1:4] * self.size[:, None]
        self.h = self.length / (2.0 ** lev)
        self.conforming, self.hanging = match_faces3(self.lo, self.size, 1 << self.lmax)

    @property
    def n_elem(self) -> int:
        return len(self.cells)


def match_faces3(lo: np.ndarray, size: np.ndarray, D: int):
    """All face couplings of a periodic octree leaf list.

    Returns
      conforming: list of (A, B, d): the +d face of A meets the -d face of B, equal size.
      hanging:    list of (A, B, d, large, q1, q2): A's +d face meets B's -d face with
                  unequal sizes; ``large`` is A or B; (q1, q2) is the quadrant of the
                  large face that the small face covers (0 = lower half, 1 = upper half
                  along t1 and along t2).
    """
    conforming = []
    hanging = []
    n = len(size)
    for d in (0, 1, 2):
        t1, t2 = TANGENTIAL[d]
        minus_faces = defaultdict(list)
        for e in range(n):
            minus_faces[int(lo[e, d])].append(e)
        for A in range(n):
            plane = int((lo[A, d] + size[A]) % D)
            a1, a2 = int(lo[A, t1]), int(lo[A, t2])
            sa = int(size[A])
            for B in minus_faces[plane]:
                b1, b2 = int(lo[B, t1]), int(lo[B, t2])
                sb = int(size[B])
                o1 = min(a1 + sa, b1 + sb) - max(a1, b1)
                o2 = min(a2 + sa, b2 + sb) - max(a2, b2)
                if o1 <= 0 or o2 <= 0:
                    continue
                if sa == sb:
                    conforming.append((A, B, d))
                elif sa > sb:
                    hanging.append((A, B, d, A, int(b1 != a1), int(b2 != a2)))
                else:
                    hanging.append((A, B, d, B, int(a1 != b1), int(a2 != b2)))
    return conforming, hanging


def is_balanced3(mesh: OctreeMesh) -> bool:
    """2:1 balance across faces: every hanging coupling joins cells whose sizes differ by
    exactly 2x, and every hanging large face is covered by exactly four small faces."""
    count = defaultdict(int)
    for (A, B, d, large, q1, q2) in mesh.hanging:
        small = B if large == A else A
        if mesh.size[large] != 2 * mesh.size[small]:
            return False
        count[(large, d, large == A)] += 1
    return all(v == 4 for v in count.values())
