"""CPU tests of libperk's host side: the library loads, exports every entry
point of include/perk.h and include/perk3d.h, and its host utilities (reference nodes, disk-polynomial
tableau, quadtree connectivity) agree with the oracle."""
import os
import re

import numpy as np
import pytest

from oracle.lgl import lgl_nodes_weights
from oracle.perk import disk_polynomial_alpha, perk2_family, perk2_free_coefficients
from oracle.treemesh import TreeMesh
from perk_inputs import kh_band_cells, uniform_cells, vortex_two_level_cells

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2403_05144_gb300.build import build
    build()
    from paper_2403_05144_gb300 import _lib
    return _lib.load()


def declared_symbols():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(perk(?:3d)?_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    from paper_2403_05144_gb300._lib import SIGNATURES
    assert sorted(n for n, _, _ in SIGNATURES) == declared_symbols()


@pytest.mark.parametrize("N", [1, 2, 3, 4, 7])
def test_reference_nodes_match_oracle(lib, N):
    from paper_2403_05144_gb300 import reference_nodes
    x, w = reference_nodes(N)
    xo, wo = lgl_nodes_weights(N)
    np.testing.assert_allclose(x, xo, rtol=0, atol=2e-16)
    np.testing.assert_allclose(w, wo, rtol=0, atol=4e-16)


@pytest.mark.parametrize("E_list", [[4, 8], [8, 16], [4, 6, 10, 16], [2, 3, 5], [6]])
def test_disk_tableau_matches_oracle(lib, E_list):
    from paper_2403_05144_gb300 import perk2_disk_tableau
    c, a = perk2_disk_tableau(E_list)
    fam = perk2_family(E_list)
    np.testing.assert_allclose(c, fam.c, rtol=0, atol=1e-16)
    for r, E in enumerate(E_list):
        free = perk2_free_coefficients(fam.S, E, disk_polynomial_alpha(E))   # 1-based stage index
        # a[r, i] = a_{i+1, i} (1-based), i.e. free[i + 1]
        np.testing.assert_allclose(a[r, 1:], free[2:], rtol=2e-15, atol=0)


def _faces_as_sets(cells):
    from paper_2403_05144_gb300 import mesh_faces
    ifs, ms = mesh_faces(cells)
    conf = {(int(a), int(b), int(d)) for a, b, d, _ in ifs}
    hang = set()
    for large, s0, s1, w in ms:
        d, side = int(w & 1), int((w >> 1) & 1)
        for half, s in ((0, s0), (1, s1)):
            A, B = (int(large), int(s)) if side == 0 else (int(s), int(large))
            hang.add((A, B, d, int(large), half))
    return conf, hang, len(ifs), len(ms)


@pytest.mark.parametrize("cells_fn", [lambda: vortex_two_level_cells(), lambda: kh_band_cells(4, 7),
                                      lambda: uniform_cells(2), lambda: [(0, 0, 0)],
                                      lambda: vortex_two_level_cells(3, 2, 6)])
def test_connectivity_matches_geometric_matching(lib, cells_fn):
    cells = cells_fn()
    conf, hang, n_if, n_m = _faces_as_sets(cells)
    m = TreeMesh(cells, 0.0, 1.0)
    assert n_if == len(m.conforming) and conf == set(m.conforming)
    assert 2 * n_m == len(m.hanging) and hang == set(m.hanging)


def test_connectivity_rejects_bad_meshes(lib):
    from paper_2403_05144_gb300 import PerkError, mesh_faces
    with pytest.raises(PerkError):
        mesh_faces([(1, 0, 0), (1, 1, 0), (1, 0, 1)])                 # does not tile
    with pytest.raises(PerkError):
        mesh_faces([(1, 0, 0), (1, 1, 0), (1, 0, 1), (1, 1, 1), (1, 1, 1)])   # duplicate
    # a level-1 cell next to level-3 cells: not 2:1 balanced
    cells = [(1, 0, 0), (1, 0, 1), (1, 1, 1)]
    for ix in range(4, 8):
        for iy in range(0, 4):
            if ix < 6 or iy >= 2:
                cells.append((3, ix, iy))
    cells += [(2, 3, 0)]
    with pytest.raises(PerkError):
        mesh_faces(cells)


@pytest.mark.parametrize("E", [3, 4, 8, 16])
def test_third_order_disk_polynomial_matches_oracle(lib, E):
    from oracle.perk import disk_polynomial3_alpha
    from paper_2403_05144_gb300 import perk3_disk_alpha
    al, r = perk3_disk_alpha(E)
    alo, ro = disk_polynomial3_alpha(E)
    np.testing.assert_allclose(al, alo, rtol=1e-10, atol=1e-18)
    assert abs(r - ro) < 1e-6 * r


@pytest.mark.parametrize("E_list", [[4, 8, 16], [3, 4, 7], [3]])
def test_third_order_family_is_valid(lib, E_list):
    # several members can satisfy the conditions; check the defining ones
    from oracle.perk import disk_polynomial3_alpha, perk3_abscissae, perk3_weights, stability_polynomial
    from paper_2403_05144_gb300 import perk3_disk_tableau
    c, a = perk3_disk_tableau(E_list)
    S = len(c)
    np.testing.assert_allclose(c, perk3_abscissae(S), atol=1e-16)
    b = perk3_weights(S)
    for r, E in enumerate(E_list):
        A = np.zeros((S, S))
        for i in range(1, S):
            A[i, i - 1] += a[r, i]
            A[i, 0] += c[i] - a[r, i]
        assert np.all(a[r] >= 0) and np.all(c - a[r] >= -1e-16)
        assert abs(b @ A @ c - 1 / 6) < 1e-13
        P = stability_polynomial(A, b)
        np.testing.assert_allclose(P[:E + 1], disk_polynomial3_alpha(E)[0], rtol=1e-9, atol=1e-18)
        assert np.all(np.abs(P[E + 1:]) < 1e-18)


@pytest.mark.parametrize("b_S", [0.5, 0.75])
def test_weighted_disk_tableau_matches_oracle(lib, b_S):
    from paper_2403_05144_gb300 import perk2_disk_tableau
    E = [4, 6, 10, 16]
    c, a = perk2_disk_tableau(E, b_S=b_S)
    fam = perk2_family(E, b_S=b_S)
    np.testing.assert_allclose(c, fam.c, rtol=1e-15, atol=0)
    for r, e in enumerate(E):
        free = perk2_free_coefficients(fam.S, e, disk_polynomial_alpha(e), b_S)   # 1-based stage index
        np.testing.assert_allclose(a[r, 1:], free[2:], rtol=2e-15, atol=0)


@pytest.mark.parametrize("E,pattern", [([4, 8, 16], "early"), ([4, 6], "alternating"), ([6, 12], "alternating"),
                                       ([4, 6, 10, 16], "classic")])
def test_pattern_tableau_matches_oracle(lib, E, pattern):
    from paper_2403_05144_gb300 import perk2_pattern_tableau
    c, ev, src, a = perk2_pattern_tableau(E, pattern)
    fam = perk2_family(E, pattern=pattern)
    np.testing.assert_allclose(c, fam.c, rtol=0, atol=1e-16)
    for r in range(len(E)):
        A = np.zeros((fam.S, fam.S))
        for i in range(1, fam.S):
            A[i, src[r, i]] += a[r, i]
            A[i, 0] += c[i] - a[r, i]
        np.testing.assert_allclose(A, fam.A[r], rtol=1e-13, atol=1e-15)
        assert [bool(x) for x in ev[r]] == [fam.active(r, i) for i in range(fam.S)]


def _balance_cases():
    rng = np.random.default_rng(41)
    cases = []
    for cells in (uniform_cells(3), vortex_two_level_cells(3, 2, 6), kh_band_cells(3, 6, 0.05)):
        lev = np.asarray(cells)[:, 0]
        for _ in range(3):
            cases.append((cells, np.clip(lev + rng.integers(-1, 2, size=len(lev)), 1, 7)))
        cases.append((cells, lev - (lev > 1)))
    return cases


@pytest.mark.parametrize("case", range(12))
def test_amr_balance_matches_the_oracle(lib, case):
    """The quadtree AMR plan's balanced levels (sibling and 2:1 rules) against the oracle's."""
    from oracle.amr import balance
    from paper_2403_05144_gb300 import amr_balance
    cells, desired = _balance_cases()[case]
    got = amr_balance(cells, desired)
    want = balance(TreeMesh(np.asarray(cells), 0.0, 1.0), desired)
    assert np.array_equal(got, want)


def test_entry_points_refuse_a_null_context(lib):
    # the calls that drive the launch structure, the adjoint and the AMR cycle check their context
    # before any CUDA call: a null context is PERK_E_INVALID_ARG, here without a GPU
    import ctypes as C
    INVALID = 1
    out_i, out_d, out_z = C.c_int32(), C.c_double(), C.c_size_t()
    calls = {
        "perk_set_stage_fusion": (None, 1),
        "perk_autotune_step": (None, None, None, C.byref(out_i)),
        "perk_autotune_volume": (None, None, C.byref(out_i)),
        "perk_adapt_commit_dt": (None, None, None, C.c_double(0.7), C.byref(out_d)),
        "perk_adapt_commit": (None, None, None),
        "perk_step_store": (None, None, C.c_double(1e-3), None),
        "perk_step_vjp_stored": (None, None, C.c_double(1e-3), None, None, None),
        "perk_step_vjp": (None, None, C.c_double(1e-3), None, None),
        "perk_workspace_bytes": (None, C.c_int64(0), C.byref(out_z)),
        "perk_bind_workspace": (None, None, C.c_size_t(0)),
        "perk_check": (None,),
    }
    for name, args in calls.items():
        assert getattr(lib, name)(*args) == INVALID, name
