"""Helpers shared by the GPU parity tests (no test functions here)."""
import numpy as np

from oracle.lgl import lgl_nodes_weights
from perk_inputs import smooth_random_state

X3, W3 = lgl_nodes_weights(3)


def discontinuous_state(cells, x0, L, seed=11, amplitude=0.2, jump=0.05):
    """Seeded smooth state with an independent per-node perturbation, so that
    element traces jump across every face."""
    U = smooth_random_state(cells, x0, L, X3, seed=seed, amplitude=amplitude)
    return U * (1.0 + jump * np.random.default_rng(seed + 1).uniform(-1, 1, size=U.shape))


def rel_err_per_var(got, want):
    """max over conserved variables of ||got - want||_inf / ||want||_inf (per variable)."""
    errs = []
    for v in range(4):
        den = max(np.max(np.abs(want[:, v])), 1e-300)
        errs.append(np.max(np.abs(got[:, v] - want[:, v])) / den)
    return max(errs)


def solver_for(cells, x0, L, flux="hll", E=None, use_graph=True):
    from paper_2403_05144_gb300 import PerkSolver
    s = PerkSolver(surface_flux=flux, use_graph=use_graph)
    s.upload_mesh(cells, x0, L)
    if E is not None:
        s.set_perk2_disk(E)
    return s
