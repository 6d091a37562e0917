"""The library's spectrum-optimised polynomials (paper_2403_05144_gb300/spectrum.py, host side)
against closed forms and against the oracle's independent optimiser (cutting-plane LPs)."""

import math

import numpy as np
import pytest

from oracle.perk import stability_polynomial
from oracle.spectrum import hull_points, optimal_polynomial

DISK = -1.0 + np.exp(1j * np.linspace(0.0, np.pi, 200)[1:])
SEGMENT = -np.linspace(0.0, 1.0, 400)[1:].astype(complex)


@pytest.fixture(scope="module")
def spec():
    from paper_2403_05144_gb300 import _lib
    from paper_2403_05144_gb300.build import build
    build()
    _lib.load()
    from paper_2403_05144_gb300 import spectrum
    return spectrum


@pytest.mark.parametrize("E,p,r", [(4, 1, 4.0), (8, 1, 8.0), (4, 2, 3.0), (8, 2, 7.0)])
def test_disk_optima(spec, E, p, r):
    dt, alpha = spec.optimize(DISK, E, p)
    assert abs(dt - r) < 1e-3 * r
    np.testing.assert_allclose(alpha[: p + 1], [1.0 / math.factorial(i) for i in range(p + 1)])


def test_chebyshev_segment(spec):
    dt, _ = spec.optimize(SEGMENT, 4, 1)
    assert abs(dt - 32.0) < 1e-3 * 32.0


@pytest.fixture(scope="module")
def dgsem_spectrum():
    # eigenvalues of the oracle's DGSEM Jacobian (Kelvin-Helmholtz state, 2x2 cells, HLLC)
    from oracle.autodiff import TorchDGSEM
    from oracle.lgl import lgl_nodes_weights
    from oracle.spectrum import dense_jacobian
    from oracle.treemesh import TreeMesh
    from perk_inputs import kelvin_helmholtz, nodal_state, uniform_cells
    x, _ = lgl_nodes_weights(3)
    cells = uniform_cells(1)
    dg = TorchDGSEM(TreeMesh(cells, -1.0, 2.0), 3, "hllc")
    U = nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, x)
    return np.linalg.eigvals(dense_jacobian(lambda V: dg.rhs(V), U))


def test_boundary_matches_oracle_hull(spec, dgsem_spectrum):
    mine = spec.boundary(dgsem_spectrum)
    ref = hull_points(dgsem_spectrum)
    key = lambda z: sorted((round(v.real, 9), round(v.imag, 9)) for v in z)
    assert key(mine) == key(ref)


@pytest.mark.parametrize("E", [4, 8])
def test_optimum_on_a_dgsem_spectrum_matches_oracle(spec, dgsem_spectrum, E):
    sigma = spec.boundary(dgsem_spectrum)
    dt, alpha = spec.optimize(sigma, E, 2)
    dt_ref, _ = optimal_polynomial(sigma, E, 2)
    assert abs(dt - dt_ref) < 1e-5 * dt_ref
    # stable at every eigenvalue with Re <= 0 (not only the hull points)
    z = dt * dgsem_spectrum[dgsem_spectrum.real <= 1e-12]
    w = np.polyval(alpha[::-1], z)
    assert np.max(np.abs(w)) <= 1.0 + 1e-8


def test_member_from_optimised_polynomial_reproduces_it(spec, dgsem_spectrum):
    # the tableau built by perk_perk2_member has the optimised polynomial as its stability polynomial
    from paper_2403_05144_gb300 import perk2_member
    S, E = 16, 8
    sigma = spec.boundary(dgsem_spectrum)
    _, alpha = spec.optimize(sigma, E, 2)
    a = perk2_member(S, E, alpha)
    c = np.arange(S) / (2.0 * (S - 1))
    A = np.zeros((S, S))
    for i in range(1, S):
        A[i, i - 1] = a[i]
        A[i, 0] = c[i] - a[i]
    b = np.zeros(S)
    b[-1] = 1.0
    coeffs = stability_polynomial(A, b)
    np.testing.assert_allclose(coeffs[: E + 1], alpha, rtol=1e-9, atol=1e-15)
    assert np.all(np.abs(coeffs[E + 1:]) < 1e-14)


def test_max_stable_dt_of_the_disk_polynomial(spec):
    E = 6
    al = [((E - 1) / E) * math.comb(E, k) / (E - 1) ** k for k in range(E + 1)]
    al[0] += 1.0 / E
    assert abs(spec.max_stable_dt(al, DISK) - (E - 1)) < 1e-6 * (E - 1)
