"""Pins of the third-order P-ERK construction (oracle): the E = 3 case is the
Shu-Osher scheme and its disk polynomial the RK3 one, every member meets the
p = 3 order conditions with shared b and c, internal consistency, the coupling
condition and positivity, and its stability polynomial equals the target."""
import math

import numpy as np
import pytest

from oracle.perk import (disk_polynomial3_alpha, perk3_abscissae, perk3_family, perk3_member, perk3_weights,
                         stability_polynomial)


def test_e3_is_rk3_and_unit_disk():
    alpha, r = disk_polynomial3_alpha(3)
    np.testing.assert_allclose(alpha, [1, 1, 0.5, 1 / 6], atol=1e-12)
    assert abs(r - 1.0) < 1e-6


def test_three_stages_is_shu_osher():
    A = perk3_member(3, 3, disk_polynomial3_alpha(3)[0])
    np.testing.assert_allclose(perk3_abscissae(3), [0, 1, 0.5])
    np.testing.assert_allclose(perk3_weights(3), [1 / 6, 1 / 6, 2 / 3])
    np.testing.assert_allclose(A, [[0, 0, 0], [1, 0, 0], [0.25, 0.25, 0]], atol=1e-12)


@pytest.mark.parametrize("E", [4, 8, 16])
def test_disk_polynomial_is_third_order_and_stable(E):
    alpha, r = disk_polynomial3_alpha(E)
    np.testing.assert_allclose(alpha[:4], [1, 1, 0.5, 1 / 6], atol=1e-12)
    th = np.linspace(0, 2 * math.pi, 721)
    z = -r + r * np.exp(1j * th)
    assert np.max(np.abs(np.polyval(alpha[::-1], z))) <= 1 + 1e-8
    assert r > 0.6 * (E - 1)


@pytest.mark.parametrize("E_list", [[4, 8, 16], [3, 4, 7], [5]])
def test_family_order_conditions(E_list):
    fam = perk3_family(E_list)
    one = np.ones(fam.S)
    assert abs(fam.b @ one - 1) < 1e-15 and abs(fam.b @ fam.c - 0.5) < 1e-15
    assert abs(fam.b @ fam.c ** 2 - 1 / 3) < 1e-15
    for E, A in zip(fam.E, fam.A):
        assert abs(fam.b @ A @ fam.c - 1 / 6) < 1e-13            # the coupling condition
        np.testing.assert_allclose(A @ one, fam.c, atol=1e-15)     # internal consistency
        assert np.all(A >= -1e-15)                                 # no downwinding
        P = stability_polynomial(A, fam.b)
        alpha = disk_polynomial3_alpha(E)[0]
        np.testing.assert_allclose(P[:E + 1], alpha, rtol=1e-9, atol=1e-18)
        assert np.all(np.abs(P[E + 1:]) < 1e-18)
