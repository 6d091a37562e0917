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

    Candidate neighbours are looked up by the position and size their -d face would have
    (equal size, half size in each of four quadrants, or the aligned double-size square); the
    overlapping areas found must cover the +d face exactly, else the mesh is not a 2:1-balanced
    tiling and ValueError is raised.
    """
    conforming = []
    hanging = []
    n = len(size)
    for d in (0, 1, 2):
        t1, t2 = TANGENTIAL[d]
        minus = {(int(lo[e, d]), int(lo[e, t1]), int(lo[e, t2]), int(size[e])): e for e in range(n)}
        for A in range(n):
            plane = int((lo[A, d] + size[A]) % D)
            a1, a2 = int(lo[A, t1]), int(lo[A, t2])
            sa = int(size[A])
            cands = [(plane, a1, a2, sa), (plane, a1 - a1 % (2 * sa), a2 - a2 % (2 * sa), 2 * sa)]
            if sa > 1:
                h = sa // 2
                cands += [(plane, a1 + i * h, a2 + j * h, h) for j in (0, 1) for i in (0, 1)]
            covered = 0
            for key in cands:
                B = minus.get(key)
                if B is None:
                    continue
                b1, b2 = int(lo[B, t1]), int(lo[B, t2])
                sb = int(size[B])
                o1 = min(a1 + sa, b1 + sb) - max(a1, b1)
                o2 = min(a2 + sa, b2 + sb) - max(a2, b2)
                if o1 <= 0 or o2 <= 0:
                    continue
                covered += o1 * o2
                if sa == sb:
                    conforming.append((A, B, d))
                elif sa > sb:
                    hanging.append((A, B, d, A, int(b1 != a1), int(b2 != a2)))
                else:
                    hanging.append((A, B, d, B, int(a1 != b1), int(a2 != b2)))
            if covered != sa * sa:
                raise ValueError(f"cell {A}: its +{d} face is not covered by 2:1-balanced neighbours")
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
