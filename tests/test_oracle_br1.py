"""Pins of the oracle's BR1 viscous terms: free stream, viscous decay and heat
conduction against the continuous operators (with convergence), conservation
at hanging faces and dissipation of kinetic energy."""
import math

import numpy as np
import pytest

from oracle.br1 import NavierStokesDGSEM
from oracle.lgl import lgl_nodes_weights
from oracle.treemesh import TreeMesh
from perk_inputs import node_coordinates, nodal_state, prim_to_cons, smooth_random_state, vortex_two_level_cells

X3, W3 = lgl_nodes_weights(3)
MU = 1e-2


def meshes():
    for lev in (3, 4):
        yield vortex_two_level_cells(lev, 2 ** (lev - 2), 3 * 2 ** (lev - 2))


def test_free_stream_has_no_viscous_terms():
    cells = vortex_two_level_cells(3, 2, 6)
    U = nodal_state(lambda X, Y: prim_to_cons(1.3 + 0 * X, 0.2 + 0 * X, -0.4 + 0 * X, 2.0 + 0 * X), cells, 0, 1, X3)
    # rounding of D w scaled twice by 2/h (~16 here)
    assert np.max(np.abs(NavierStokesDGSEM(TreeMesh(cells, 0, 1.0), mu=MU).viscous_rhs(U))) < 1e-11


def test_shear_wave_momentum_is_mu_laplacian():
    errs = []
    for cells in meshes():
        A = 0.1
        U = nodal_state(lambda X, Y: prim_to_cons(1 + 0 * X, A * np.sin(2 * math.pi * Y), 0 * X, 10 + 0 * X),
                        cells, 0, 1, X3)
        K = NavierStokesDGSEM(TreeMesh(cells, 0, 1.0), mu=MU).viscous_rhs(U)
        _, Y = node_coordinates(cells, 0, 1, X3)
        errs.append(np.max(np.abs(K[:, 1] + MU * 4 * math.pi ** 2 * A * np.sin(2 * math.pi * Y))))
        assert np.max(np.abs(K[:, 0])) == 0.0          # no viscous mass flux
    assert errs[1] < 0.5 * errs[0] and errs[1] < 1e-3


def test_heat_conduction_is_kappa_laplacian():
    # at rest with uniform density: dE/dt = kappa d2T/dx2, T = p / rho
    errs = []
    for cells in meshes():
        eps = 0.05
        U = nodal_state(lambda X, Y: prim_to_cons(1 + 0 * X, 0 * X, 0 * X, 1 + eps * np.sin(2 * math.pi * X)),
                        cells, 0, 1, X3)
        ns = NavierStokesDGSEM(TreeMesh(cells, 0, 1.0), mu=MU, prandtl=0.72)
        K = ns.viscous_rhs(U)
        X, _ = node_coordinates(cells, 0, 1, X3)
        kappa = MU * 1.4 / (0.4 * 0.72)
        errs.append(np.max(np.abs(K[:, 3] + kappa * eps * 4 * math.pi ** 2 * np.sin(2 * math.pi * X))))
    assert errs[1] < 0.5 * errs[0] and errs[1] < 2e-3


def test_conservation_and_dissipation_on_hanging_faces():
    cells = vortex_two_level_cells(3, 2, 6)
    m = TreeMesh(cells, 0, 1.0)
    U = smooth_random_state(cells, 0, 1.0, X3, amplitude=0.2)
    U = U * (1 + 0.05 * np.random.default_rng(3).uniform(-1, 1, U.shape))
    ns = NavierStokesDGSEM(m, mu=MU)
    K = ns.viscous_rhs(U)
    assert np.all(np.abs(ns.integrate(K)) < 1e-14 * np.max(np.abs(K)))
    # kinetic energy change by the viscous terms at uniform temperature: v . dm - |v|^2/2 drho <= 0
    Uc = nodal_state(lambda X, Y: prim_to_cons(1 + 0 * X, 0.3 * np.sin(2 * math.pi * (X + Y)),
                                               0.2 * np.cos(2 * math.pi * X), 2 + 0 * X), cells, 0, 1, X3)
    K = ns.viscous_rhs(Uc)
    v1, v2 = Uc[:, 1] / Uc[:, 0], Uc[:, 2] / Uc[:, 0]
    dke = v1 * K[:, 1] + v2 * K[:, 2] - 0.5 * (v1 ** 2 + v2 ** 2) * K[:, 0]
    assert np.einsum("e,eji,ji->", (0.5 * m.h) ** 2, dke, np.outer(W3, W3)) < 0.0
