"""Pins of the oracle's differentiable transcription: equal to the numpy oracle,
its JVP equal to central differences of the numpy oracle, the dot-product
identity between its forward and reverse modes, and the step adjoint against
central differences."""
import numpy as np
import pytest
import torch

from oracle.autodiff import TorchDGSEM, jvp_rhs, perk_step_torch, vjp_rhs, vjp_steps
from oracle.dgsem import DGSEM
from oracle.lgl import lgl_nodes_weights
from oracle.perk import element_methods, perk2_family, prkm_step
from oracle.treemesh import TreeMesh
from perk_inputs import smooth_random_state, vortex_two_level_cells

X3, _ = lgl_nodes_weights(3)
CELLS = vortex_two_level_cells(2, 1, 3)


def state():
    U = smooth_random_state(CELLS, -1.0, 2.0, X3, amplitude=0.2)
    return U * (1 + 0.05 * np.random.default_rng(1).uniform(-1, 1, U.shape))


@pytest.mark.parametrize("flux", ["hll", "hllc", "ec"])
def test_transcription_equals_numpy_oracle(flux):
    m = TreeMesh(CELLS, -1.0, 2.0)
    U = state()
    K = DGSEM(m, 3, flux).rhs(U)
    Kt = TorchDGSEM(m, 3, flux).rhs(torch.tensor(U)).numpy()
    assert np.max(np.abs(K - Kt)) < 1e-13 * np.max(np.abs(K))


@pytest.mark.parametrize("flux", ["hll", "hllc"])
def test_jvp_vs_central_differences_and_dot_product(flux):
    m = TreeMesh(CELLS, -1.0, 2.0)
    U = state()
    rng = np.random.default_rng(3)
    v, w = rng.normal(size=U.shape), rng.normal(size=U.shape)
    dg = TorchDGSEM(m, 3, flux)
    jv = jvp_rhs(dg, U, v)
    eps = 1e-6
    rhs = DGSEM(m, 3, flux).rhs
    fd = (rhs(U + eps * v) - rhs(U - eps * v)) / (2 * eps)
    # the steep shear layer on 28 cells makes the central difference itself
    # accurate to ~5e-7 only; a wrong tie derivative is off by ~1e-2
    assert np.max(np.abs(fd - jv)) < 2e-6 * np.max(np.abs(jv))
    jt = vjp_rhs(dg, U, w)
    assert abs(np.sum(jv * w) - np.sum(v * jt)) < 1e-12 * np.sum(np.abs(jv * w))


def test_step_adjoint_vs_central_differences():
    m = TreeMesh(CELLS, -1.0, 2.0)
    U = state()
    fam = perk2_family([4, 8])
    meth = element_methods(m.cells[:, 0], fam.R)
    dt = 0.01
    rng = np.random.default_rng(4)
    lam, d = rng.normal(size=U.shape), rng.normal(size=U.shape)
    g = vjp_steps(TorchDGSEM(m, 3, "hll"), U, lam, dt, fam, meth, 2)
    rhs = DGSEM(m, 3, "hll").rhs

    def F(X):
        for _ in range(2):
            X = prkm_step(rhs, X, dt, fam, meth)
        return np.sum(lam * X)

    eps = 1e-6
    fd = (F(U + eps * d) - F(U - eps * d)) / (2 * eps)
    assert abs(fd - np.sum(g * d)) < 1e-7 * abs(fd)
    # the torch step equals the numpy step
    Ut = perk_step_torch(TorchDGSEM(m, 3, "hll"), torch.tensor(U), dt, fam, meth).numpy()
    assert np.max(np.abs(Ut - prkm_step(rhs, U, dt, fam, meth))) < 1e-13


def test_derivatives_at_tied_arguments():
    # the continuous Kelvin-Helmholtz state has exactly equal neighbouring values
    # (density depends on y only, unit pressure): the logarithmic mean must be
    # differentiated through its smooth series there, not through a tie branch
    from perk_inputs import kelvin_helmholtz, nodal_state
    m = TreeMesh(CELLS, -1.0, 2.0)
    U = nodal_state(kelvin_helmholtz, CELLS, -1.0, 2.0, X3)
    assert np.any(U[:, 0, :, 0] == U[:, 0, :, 1])          # ties present
    rng = np.random.default_rng(6)
    v, w = rng.normal(size=U.shape), rng.normal(size=U.shape)
    dg = TorchDGSEM(m, 3, "hllc")
    jv = jvp_rhs(dg, U, v)
    rhs = DGSEM(m, 3, "hllc").rhs
    eps = 1e-6
    fd = (rhs(U + eps * v) - rhs(U - eps * v)) / (2 * eps)
    # the steep shear layer on 28 cells makes the central difference itself
    # accurate to ~5e-7 only; a wrong tie derivative is off by ~1e-2
    assert np.max(np.abs(fd - jv)) < 2e-6 * np.max(np.abs(jv))
    jt = vjp_rhs(dg, U, w)
    assert abs(np.sum(jv * w) - np.sum(v * jt)) < 1e-12 * np.sum(np.abs(jv * w))
