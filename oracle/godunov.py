"""1D upwind finite-volume model problem (oracle; test infrastructure only).

Sec. 3.2.1 of the paper applies a two-member P-ERK scheme to
u_t + u_x = 0 on (-1, 1), periodic, discretised by the first-order upwind
(Godunov) scheme, Eq. UpwindFullSystem:  dU_i/dt = (U_{i-1} - U_i) / dx_i.
Being linear, one step is a matrix D (Eq. PartitionedSystem) whose columns
are the step applied to unit vectors.
"""

from __future__ import annotations

import numpy as np

from .perk import PERKFamily, perk2_family, prkm_step


def upwind_operator(dx: np.ndarray) -> np.ndarray:
    """L with L[i, i] = -1/dx_i and L[i, i-1] = +1/dx_i (periodic: L[0, N-1])."""
    n = len(dx)
    L = np.zeros((n, n))
    for i in range(n):
        L[i, i] = -1.0 / dx[i]
        L[i, (i - 1) % n] = 1.0 / dx[i]
    return L


def two_region_grid(n_coarse: int, alpha: float):
    """Cells of (-1, 1) with dx_1 = 2 / n_coarse outside [-0.5, 0.5] and
    dx_1 / alpha inside.  Returns (cell edges, dx, fine-region mask)."""
    dx1 = 2.0 / n_coarse
    n_side = n_coarse // 4                               # cells in (-1, -0.5] and in [0.5, 1)
    n_mid = int(round(alpha * n_coarse / 2))              # cells in [-0.5, 0.5]
    dx = np.concatenate([np.full(n_side, dx1), np.full(n_mid, 1.0 / n_mid), np.full(n_side, dx1)])
    edges = np.concatenate([[-1.0], -1.0 + np.cumsum(dx)])
    fine = np.zeros(len(dx), dtype=bool)
    fine[n_side:n_side + n_mid] = True
    return edges, dx, fine


def cell_averages(edges: np.ndarray) -> np.ndarray:
    """Exact cell averages of u0 = 1 + sin(pi x) / 2."""
    xl, xr = edges[:-1], edges[1:]
    return 1.0 + (np.cos(np.pi * xl) - np.cos(np.pi * xr)) / (2.0 * np.pi * (xr - xl))


def step_matrix(L: np.ndarray, dt: float, fam: PERKFamily, method: np.ndarray) -> np.ndarray:
    """D such that U_{n+1} = D U_n for one P-ERK step on U' = L U."""
    n = L.shape[0]

    def rhs(Y):                       # Y: [n_cells, 1, 1, n_columns]
        return (L @ Y[:, 0, 0, :])[:, None, None, :]

    Id = np.eye(n)[:, None, None, :]
    return prkm_step(rhs, Id, dt, fam, method)[:, 0, 0, :]


def total_variation(U: np.ndarray) -> float:
    """sum_i |U_{i+1} - U_i| over the periodic grid."""
    return float(np.sum(np.abs(np.roll(U, -1) - U)))


def tv_increase(n_coarse: int, alpha: float, E1: int, E2: int, cfl: float = 1.0, pattern: str = "classic") -> float:
    """Relative total-variation increase after one step with the coarse cells
    on member E1 and the refined cells on member E2, dt = cfl * (E1 - 1) * dx_1
    (the largest stable step of the E1 disk polynomial on the coarse cells);
    stage pattern classic, alternating or early (Sec. 3.2.4)."""
    edges, dx, fine = two_region_grid(n_coarse, alpha)
    fam = perk2_family([E1, E2], pattern=pattern)
    method = fine.astype(np.int64)
    dt = cfl * (E1 - 1) * dx[0]
    U0 = cell_averages(edges)

    def rhs(Y):                       # (U_{i-1} - U_i) / dx_i without forming L
        y = Y[:, 0, 0, 0]
        return ((np.roll(y, 1) - y) / dx)[:, None, None, None]

    U1 = prkm_step(rhs, U0[:, None, None, None], dt, fam, method)[:, 0, 0, 0]
    tv0 = total_variation(U0)
    return (total_variation(U1) - tv0) / tv0


def uniform_family_matrix(n: int = 64, E=(8, 16)):
    """The paper's uniform example: dx = 2/n, member E[1] in [-0.5, 0.5], E[0]
    elsewhere, dt = 0.21875 (for n = 64).  Returns (D, dt, method)."""
    edges, dx, fine = two_region_grid(n, 1.0)
    fam = perk2_family(list(E))
    method = fine.astype(np.int64)
    dt = (E[0] - 1) * dx[0]
    return step_matrix(upwind_operator(dx), dt, fam, method), dt, method
