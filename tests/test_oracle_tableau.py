"""Pins of the oracle's P-ERK2 construction: the paper's printed coefficients,
order conditions, internal consistency and the stability polynomial."""
import os

import numpy as np
import pytest

from oracle.perk import (disk_polynomial_alpha, perk2_family, perk2_free_coefficients, stability_polynomial)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "perk2_S16_E8_E16.txt")


def load_golden():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        i, c, a8, a16 = line.split()
        num, den = c.split("/")
        rows.append((int(i), float(num) / float(den), float(a8), float(a16)))
    return rows


def test_printed_table_reproduced():
    fam = perk2_family([8, 16])
    a8_free = perk2_free_coefficients(16, 8, disk_polynomial_alpha(8))
    a16_free = perk2_free_coefficients(16, 16, disk_polynomial_alpha(16))
    rows = load_golden()
    assert len(rows) == 16
    for (i, c, a8, a16) in rows:
        assert abs(fam.c[i - 1] - c) < 1e-16
        # the printed digits carry the paper's own last-bit rounding: allow a few ulp
        assert abs(a8_free[i] - a8) <= 1e-15 * a8
        assert abs(a16_free[i] - a16) <= 1e-15 * a16
        if i >= 3:
            # the dense arrays carry the same entries below the diagonal ...
            assert fam.A[0][i - 1, i - 2] == a8_free[i] and fam.A[1][i - 1, i - 2] == a16_free[i]
        if i >= 2:
            # ... and a_{i,1} = c_i - a_{i,i-1}
            assert abs(fam.A[1][i - 1, 0] + (a16_free[i] if i >= 3 else 0.0) - c) < 1e-16


@pytest.mark.parametrize("E_list", [[8, 16], [4, 8], [4, 6, 10, 16], [2, 3], [5]])
def test_order_conditions_and_consistency(E_list):
    fam = perk2_family(E_list)
    ones = np.ones(fam.S)
    assert abs(fam.b @ ones - 1.0) < 1e-15                  # p = 1
    assert abs(fam.b @ fam.c - 0.5) < 1e-15                 # p = 2
    for A in fam.A:
        np.testing.assert_allclose(A @ ones, fam.c, atol=1e-15)   # internal consistency
        assert np.all(np.triu(A) == 0.0)                     # explicit
        # only K_1 and K_{i-1} enter stage i
        for i in range(fam.S):
            nz = np.nonzero(A[i])[0]
            assert set(nz.tolist()) <= {0, i - 1}


@pytest.mark.parametrize("E", [2, 3, 4, 6, 8, 10, 16])
@pytest.mark.parametrize("S_extra", [0, 3])
def test_stability_polynomial_matches_alpha(E, S_extra):
    S = E + S_extra
    fam = perk2_family([E], S=S)
    P = stability_polynomial(fam.A[0], fam.b)
    alpha = disk_polynomial_alpha(E)
    np.testing.assert_allclose(P[:E + 1], alpha, rtol=1e-13, atol=1e-17)
    assert np.all(np.abs(P[E + 1:]) < 1e-17)                 # degree E exactly: E evaluations


@pytest.mark.parametrize("E", [3, 4, 8, 16])
def test_disk_polynomial_stability_and_radius(E):
    alpha = disk_polynomial_alpha(E)
    r = E - 1.0
    th = np.linspace(0, 2 * np.pi, 721)
    z = -r + r * np.exp(1j * th)
    # the monomial form loses ~1e-10 to cancellation at |z| ~ 2(E-1), hence the tolerance
    assert np.max(np.abs(np.polyval(alpha[::-1], z))) <= 1.0 + 1e-8
    # the second-order consistency of the closed form
    assert alpha[0] == pytest.approx(1.0, abs=1e-15)
    assert alpha[1] == pytest.approx(1.0, abs=1e-15)
    assert alpha[2] == pytest.approx(0.5, abs=1e-15)
    # a slightly larger disk leaves the stability region
    zz = -1.02 * r + 1.02 * r * np.exp(1j * th)
    assert np.max(np.abs(np.polyval(alpha[::-1], zz))) > 1.0 + 1e-3


def test_free_coefficients_are_zero_before_first_shared_stage():
    a = perk2_free_coefficients(16, 8, disk_polynomial_alpha(8))
    assert np.all(a[:11] == 0.0) and np.all(a[11:] > 0.0)


@pytest.mark.parametrize("b_S,c2", [(0.5, 1.0), (0.75, 2.0 / 3.0)])
def test_two_stage_weight_variants_are_heun_and_ralston(b_S, c2):
    # S = E = 2 with b_1 = 1 - b_S: Heun's method (b = (1/2, 1/2), c_2 = 1) and Ralston's
    # (b = (1/4, 3/4), c_2 = 2/3), the variants named in Sec. 3.1
    from oracle.perk import perk2_family
    fam = perk2_family([2], b_S=b_S)
    np.testing.assert_allclose(fam.b, [1.0 - b_S, b_S], rtol=0, atol=1e-16)
    np.testing.assert_allclose(fam.c, [0.0, c2], rtol=0, atol=1e-16)
    np.testing.assert_allclose(fam.A[0], [[0.0, 0.0], [c2, 0.0]], rtol=0, atol=1e-16)


@pytest.mark.parametrize("b_S", [0.5, 0.75])
def test_weight_variants_keep_order_and_polynomial(b_S):
    from oracle.perk import disk_polynomial_alpha, perk2_family, stability_polynomial
    fam = perk2_family([4, 8, 16], b_S=b_S)
    for r, E in enumerate(fam.E):
        A = fam.A[r]
        assert abs(fam.b.sum() - 1.0) < 1e-15 and abs(fam.b @ fam.c - 0.5) < 1e-15
        np.testing.assert_allclose(A.sum(axis=1), fam.c, rtol=0, atol=1e-15)
        P = stability_polynomial(A, fam.b)
        np.testing.assert_allclose(P[: E + 1], disk_polynomial_alpha(E), rtol=1e-11, atol=1e-15)
        assert np.all(np.abs(P[E + 1:]) < 1e-12)


@pytest.mark.parametrize("pattern,stages,couplings", [
    ("alternating", [1, 3, 4, 6], [(4, 3), (6, 4)]),       # Eq. PERK_ButcherTableauAlternating
    ("early", [1, 2, 3, 6], [(3, 2), (6, 3)]),             # Eq. PERK_ButcherTableauEarlyShared
    ("classic", [1, 4, 5, 6], [(5, 4), (6, 5)]),           # Eq. PERK_ButcherTableauClassic, A^(1)
])
def test_stage_patterns_reproduce_the_printed_tableaux(pattern, stages, couplings):
    # the S = 6, E = 4 member of the paper's examples: evaluated stages and the nonzero
    # entries off the first column
    from oracle.perk import pattern_stages
    fam = perk2_family([4, 6], pattern=pattern)
    assert pattern_stages(6, 4, pattern) == stages
    A = fam.A[0]
    off = {(i + 1, j + 1) for i in range(6) for j in range(1, 6) if A[i, j] != 0.0}
    assert off == set(couplings)
    np.testing.assert_allclose(A.sum(axis=1), fam.c, rtol=0, atol=1e-15)
    assert [i + 1 for i in range(6) if fam.active(0, i)] == stages


@pytest.mark.parametrize("pattern", ["alternating", "early"])
def test_stage_patterns_keep_polynomial_and_order(pattern):
    fam = perk2_family([4, 8, 16], pattern=pattern)
    for r, E in enumerate(fam.E):
        P = stability_polynomial(fam.A[r], fam.b)
        np.testing.assert_allclose(P[: E + 1], disk_polynomial_alpha(E), rtol=1e-11, atol=1e-15)
        assert np.all(np.abs(P[E + 1:]) < 1e-12)
        assert abs(fam.b @ fam.c - 0.5) < 1e-15
        # a member only couples to stages it evaluates
        ev = [i for i in range(fam.S) if fam.active(r, i)]
        for i in range(fam.S):
            for j in range(1, fam.S):
                if fam.A[r][i, j] != 0.0:
                    assert j in ev and i in ev


def test_stage_pattern_total_variation_trend():
    # Sec. 3.2.4: the stage pattern changes the nonlinear behaviour at the scheme interfaces; on
    # the 1D bench (6-12 family) the classic pattern increases the total variation least and the
    # alternating one most (trend only: the paper prints no numbers for this comparison)
    from oracle.godunov import tv_increase
    for alpha, cfl in ((1.5, 1.0), (1.5, 0.8), (2.0, 0.8)):
        tv = {p: tv_increase(64, alpha, 6, 12, cfl, p) for p in ("classic", "alternating", "early")}
        assert tv["classic"] < tv["early"] < tv["alternating"]
