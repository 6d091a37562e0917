"""Pins of the spectrum-optimised stability polynomials (oracle/spectrum.py) against
classical optima that have closed forms:

* the disk D_r = {|z + r| <= r}: the largest r for a degree-E polynomial of order 1 is E,
  attained by (1 + z/E)^E; for order 2 it is E - 1 (Jeltsch & Nevanlinna's bound
  r <= E - p + 1, attained for p <= 2);
* the real segment [-r, 0] at order 1: r = 2 E^2, attained by the shifted Chebyshev
  polynomial T_E(1 + z/E^2).
"""

import math

import numpy as np
import pytest

from oracle.spectrum import dense_jacobian, hull_points, optimal_polynomial, polynomial_values

DISK = -1.0 + np.exp(1j * np.linspace(0.0, np.pi, 200)[1:])       # |lambda + 1| = 1, upper half
SEGMENT = -np.linspace(0.0, 1.0, 400)[1:].astype(complex)          # [-1, 0)


@pytest.mark.parametrize("E,p,r", [(4, 1, 4.0), (8, 1, 8.0), (4, 2, 3.0), (8, 2, 7.0)])
def test_disk_optimum(E, p, r):
    dt, alpha = optimal_polynomial(DISK, E, p)
    assert abs(dt - r) < 1e-3 * r
    # the polynomial is stable on the constraint set (and its conjugate)
    w = polynomial_values(dt * np.concatenate([DISK, DISK.conj()]), p, alpha)
    assert np.max(np.abs(w)) <= 1.0 + 1e-9


def test_order_one_disk_polynomial_is_the_binomial():
    E = 4
    dt, alpha = optimal_polynomial(DISK, E, 1)
    want = [math.comb(E, k) / E ** k for k in range(2, E + 1)]
    np.testing.assert_allclose(alpha, want, rtol=2e-3)


@pytest.mark.parametrize("E", [2, 4])
def test_real_segment_chebyshev_optimum(E):
    dt, alpha = optimal_polynomial(SEGMENT, E, 1)
    assert abs(dt - 2 * E * E) < 1e-3 * 2 * E * E


def test_third_order_disk_is_below_the_second_order_bound():
    dt3, _ = optimal_polynomial(DISK, 8, 3)
    dt2, _ = optimal_polynomial(DISK, 8, 2)
    assert dt3 < dt2 and dt3 <= 8 - 3 + 1


def test_hull_points_of_a_grid():
    # points of a grid in the second quadrant: the hull is the rectangle's corners,
    # refined so that neighbours are no farther apart than the mean edge length
    re, im = np.meshgrid(np.linspace(-4.0, 0.0, 9), np.linspace(0.0, 1.0, 5))
    pts = (re + 1j * im).ravel()
    h = hull_points(np.concatenate([pts, pts.conj(), [1.0 + 0j]]))   # the right half plane is ignored
    corners = {complex(-4, 0), complex(-4, 1), complex(0, 1), complex(0, 0)}
    assert corners <= {complex(round(z.real, 12), round(z.imag, 12)) for z in h}
    assert np.all(h.real <= 1e-12) and np.all(h.imag >= 0)
    ring = np.concatenate([h, h[:1]])
    gaps = np.abs(np.diff(ring))
    assert gaps.max() <= np.mean([4.0, 1.0, 4.0, 1.0]) + 1e-12


def test_dense_jacobian_of_a_linear_map():
    A = np.random.default_rng(3).normal(size=(6, 6))

    def rhs(U):
        import torch
        return torch.tensor(A) @ U.reshape(-1)

    np.testing.assert_allclose(dense_jacobian(rhs, np.zeros(6)), A, rtol=0, atol=1e-15)


def test_cfl_reading_of_the_disk_polynomials():
    # the stable CFL of member E (time-step rule of the runs) on the dense spectrum of the
    # oracle's Jacobian: 2 x 2 periodic cells, N = 3, HLLC, smooth seeded state, modes with
    # Re > 0 left out; the numbers recorded as a reading of Sec. 4.1
    from oracle.autodiff import TorchDGSEM
    from oracle.lgl import lgl_nodes_weights
    from oracle.perk import disk_polynomial_alpha, max_wave_speed_dt
    from oracle.treemesh import TreeMesh
    from perk_inputs import smooth_random_state, uniform_cells
    x, _ = lgl_nodes_weights(3)
    cells = uniform_cells(1)
    m = TreeMesh(cells, -1.0, 2.0)
    U = smooth_random_state(cells, -1.0, 2.0, x)
    ev = np.linalg.eigvals(dense_jacobian(lambda V: TorchDGSEM(m, 3, "hllc").rhs(V), U))
    ev = ev[ev.real <= 1e-12]
    dt1 = max_wave_speed_dt(U, m.h, 3, 1.0)
    for E, cfl in ((4, 1.15), (16, 2.25)):
        al = disk_polynomial_alpha(E)
        modulus = lambda c: np.max(np.abs(np.polyval(al[::-1], c * dt1 * ev)))
        assert modulus(0.99 * cfl) <= 1.0 + 1e-10 < modulus(1.01 * cfl)
