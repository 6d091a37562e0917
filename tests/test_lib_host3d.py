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


def _plan_cases():
    from perk_inputs.octree import block_refined_cells3, refine_cells3, uniform_cells3
    rng = np.random.default_rng(31)
    three = refine_cells3(refine_cells3(uniform_cells3(2), lambda l, ix, iy, iz: 1 <= ix < 3 and iy < 2 and 1 <= iz),
                          lambda l, ix, iy, iz: l == 3 and 3 <= ix < 5 and 1 <= iy < 3 and 3 <= iz < 5)
    cases = []
    for cells in (uniform_cells3(2), block_refined_cells3(2, 1, 3), three):
        lev = np.asarray(cells)[:, 0]
        for _ in range(3):
            cases.append((cells, np.clip(lev + rng.integers(-1, 2, size=len(lev)), 1, 5)))
        cases.append((cells, lev - (lev > 1)))        # every cell asks to coarsen
    return cases


@pytest.mark.parametrize("case", range(12))
def test_amr_plan_matches_the_oracle(lib, case):
    """Balanced levels, new leaves (Morton order) and transfer records of the library's octree AMR
    plan against the oracle's balance and new leaves (Sec. 7.1.3's AMR cycle)."""
    from oracle.amr3d import balance3, new_cells3
    from paper_2403_05144_gb300.perk3d import amr_plan_cells
    cells, desired = _plan_cases()[case]
    mesh = OctreeMesh(np.asarray(cells), 0.0, 1.0)
    levels, new, mp = amr_plan_cells(cells, desired)
    want_levels = balance3(mesh, desired)
    assert np.array_equal(levels, want_levels)
    want_cells = new_cells3(mesh, want_levels)
    assert [tuple(c) for c in new.tolist()] == [tuple(c) for c in want_cells]
    old = {tuple(c): e for e, c in enumerate(cells)}
    for (l, x, y, z), r in zip(new.tolist(), mp.tolist()):
        kind = r[0] & 3
        if kind == 0:
            assert old[(l, x, y, z)] == r[1]
        elif kind == 1:
            assert old[(l - 1, x >> 1, y >> 1, z >> 1)] == r[1]
            assert ((r[0] >> 2) & 1, (r[0] >> 3) & 1, (r[0] >> 4) & 1) == (x & 1, y & 1, z & 1)
        else:
            for ch in range(8):
                assert old[(l + 1, 2 * x + (ch & 1), 2 * y + ((ch >> 1) & 1), 2 * z + (ch >> 2))] == r[1 + ch]


def test_amr_plan_rejects_jumps_of_two_levels(lib):
    from paper_2403_05144_gb300._lib import PerkError
    from paper_2403_05144_gb300.perk3d import amr_plan_cells
    cells = uniform_cells3(2)
    d = np.full(len(cells), 2)
    d[0] = 4
    with pytest.raises(PerkError, match="at most one"):
        amr_plan_cells(cells, d)


@pytest.mark.parametrize("seed", range(6))
def test_connectivity_of_random_balanced_octrees(lib, seed):
    """Random meshes grown by the oracle's balanced AMR cycle (random wishes, three cycles from
    level 1): the library's interfaces and mortars equal the oracle's geometric face matching."""
    from oracle.amr3d import balance3, new_cells3
    from paper_2403_05144_gb300.perk3d import mesh_faces3
    rng = np.random.default_rng(100 + seed)
    cells = uniform_cells3(1)
    for _ in range(3):
        mesh = OctreeMesh(np.asarray(cells), 0.0, 1.0)
        lev = mesh.cells[:, 0]
        wish = np.clip(lev + rng.choice([-1, 0, 1], size=len(lev), p=[0.2, 0.5, 0.3]), 0, 4)
        cells = new_cells3(mesh, balance3(mesh, wish))
    mesh = OctreeMesh(np.asarray(cells), 0.0, 1.0)
    ifs, morts = mesh_faces3(cells)
    assert sorted(map(tuple, ifs[:, :3].tolist())) == sorted(mesh.conforming)
    want = {}
    for (A, B, d, large, q1, q2) in mesh.hanging:
        want.setdefault((large, d, 0 if large == A else 1), {})[q1 + 2 * q2] = B if large == A else A
    got = {(l, f & 3, (f >> 2) & 1): {0: a, 1: b, 2: c, 3: e} for (l, a, b, c, e, f) in morts.tolist()}
    assert got == want
