"""CPU tests of the 3D host side: the octree connectivity the library builds (interfaces,
face mortars with four small cells by quadrant) equals the oracle's geometric face matching,
and malformed meshes are rejected."""
import numpy as np
import pytest

from oracle.octree import OctreeMesh
from perk_inputs.octree import block_refined_cells3, refine_cells3, slab_cells3, uniform_cells3


@pytest.fixture(scope="module")
def lib():
    from paper_2403_05144_gb300.build import build
    build()
    from paper_2403_05144_gb300 import _lib
    return _lib.load()


def _asymmetric():
    return refine_cells3(uniform_cells3(2), lambda l, ix, iy, iz: 1 <= ix < 2 and 0 <= iy < 3 and 2 <= iz < 4)


@pytest.mark.parametrize("cells_fn", [lambda: uniform_cells3(2), lambda: block_refined_cells3(2, 1, 3), _asymmetric,
                                      lambda: slab_cells3(2, 4, 1.0 / 16.0), lambda: uniform_cells3(0)])
def test_connectivity_matches_oracle(lib, cells_fn):
    from paper_2403_05144_gb300.perk3d import mesh_faces3
    cells = cells_fn()
    ifs, morts = mesh_faces3(cells)
    mesh = OctreeMesh(np.asarray(cells), 0.0, 1.0)
    assert sorted(map(tuple, ifs[:, :3].tolist())) == sorted(mesh.conforming)
    # oracle: one record per (small, large) coupling with its quadrant; library: one per large face
    want = {}
    for (A, B, d, large, q1, q2) in mesh.hanging:
        small = B if large == A else A
        side = 0 if large == A else 1
        want.setdefault((large, d, side), {})[q1 + 2 * q2] = small
    got = {}
    for (large, s0, s1, s2, s3, flags) in morts.tolist():
        got[(large, flags & 3, (flags >> 2) & 1)] = {0: s0, 1: s1, 2: s2, 3: s3}
    assert got == want


def test_rejects_unbalanced_and_untiled_meshes(lib):
    from paper_2403_05144_gb300._lib import PerkError
    from paper_2403_05144_gb300.perk3d import mesh_faces3
    # a level-3 block beside level-1 cells: 4:1 across a face
    cells = refine_cells3(refine_cells3(uniform_cells3(1), lambda l, ix, iy, iz: (ix, iy, iz) == (0, 0, 0)),
                          lambda l, ix, iy, iz: l == 2 and (ix, iy, iz) == (1, 1, 1))
    with pytest.raises(PerkError, match="balanced"):
        mesh_faces3(cells)
    with pytest.raises(PerkError, match="tile|gap"):
        mesh_faces3(uniform_cells3(1)[:-1])
    with pytest.raises(PerkError, match="duplicated"):
        mesh_faces3(uniform_cells3(1) + [uniform_cells3(1)[0]])
