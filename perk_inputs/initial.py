"""Analytic initial states of the synthetic workloads and seeded draws.

Every function here returns primitive or conserved variables of the 2D Euler
equations at given physical points; nothing here discretises anything.  The
nodal state of an element is the initial condition sampled at the element's
collocation nodes, whose reference positions the caller supplies (each side
computes its own nodes).
"""

from __future__ import annotations

import math
from typing import Sequence

import numpy as np

GAMMA = 1.4
SEED = 20240308  # default seed; each workload adds its own offset


def prim_to_cons(rho, v1, v2, p, gamma: float = GAMMA):
    return np.stack([rho, rho * v1, rho * v2, p / (gamma - 1.0) + 0.5 * rho * (v1 * v1 + v2 * v2)])


def isentropic_vortex(x, y, t: float = 0.0, *, eps: float = 5.0, u_inf: float = 1.0, v_inf: float = 1.0,
                      half_width: float = 10.0, gamma: float = GAMMA):
    """Shu's isentropic vortex on the periodic square [-half_width, half_width]^2
    (strength ``eps``, background density and pressure 1, background velocity
    (u_inf, v_inf)), translated to time ``t``; returns conserved variables."""
    L = 2.0 * half_width
    xc = u_inf * t
    yc = v_inf * t
    dx = (x - xc + half_width) % L - half_width
    dy = (y - yc + half_width) % L - half_width
    r2 = dx * dx + dy * dy
    f = np.exp(0.5 * (1.0 - r2))
    T = 1.0 - (gamma - 1.0) * eps * eps / (8.0 * gamma * math.pi ** 2) * f * f
    rho = T ** (1.0 / (gamma - 1.0))
    v1 = u_inf - eps / (2.0 * math.pi) * f * dy
    v2 = v_inf + eps / (2.0 * math.pi) * f * dx
    p = rho ** gamma
    return prim_to_cons(rho, v1, v2, p, gamma)


def kelvin_helmholtz(x, y, *, amplitude: float = 0.1, wavenumber: int = 2, gamma: float = GAMMA):
    """Kelvin-Helmholtz initial state on [-1, 1]^2: a dense band |y| < 0.5
    moving against a light background, density 0.5 + 0.75 B(y), velocity
    0.5 (B - 1), a transverse perturbation ``amplitude * sin(wavenumber*pi*x)``
    and unit pressure, with B(y) = tanh(15y + 7.5) - tanh(15y - 7.5)."""
    B = np.tanh(15.0 * y + 7.5) - np.tanh(15.0 * y - 7.5)
    rho = 0.5 + 0.75 * B
    v1 = 0.5 * (B - 1.0)
    v2 = amplitude * np.sin(wavenumber * math.pi * x)
    p = np.ones_like(rho)
    return prim_to_cons(rho, v1, v2, p, gamma)


def shear_layer(x, y, *, kappa: float = 80.0, delta: float = 0.05, mach: float = 0.3, gamma: float = GAMMA):
    """Doubly periodic shear layer on [0, 1]^2 with unit density, tanh velocity
    profiles of steepness ``kappa`` at y = 0.25 and 0.75, a transverse
    perturbation ``delta * sin(2 pi (x + 0.25))`` and the pressure of sound
    speed 1/mach."""
    v1 = np.where(y <= 0.5, np.tanh(kappa * (y - 0.25)), np.tanh(kappa * (0.75 - y)))
    v2 = delta * np.sin(2.0 * math.pi * (x + 0.25))
    rho = np.ones_like(x)
    p = rho / (gamma * mach * mach)
    return prim_to_cons(rho, v1, v2, p, gamma)


def node_coordinates(cells: Sequence, x0: float, length: float, xi: np.ndarray):
    """Physical coordinates of the tensor-product nodes of every cell.

    ``xi`` are the 1D reference nodes on [-1, 1].  Returns ``(X, Y)`` of shape
    ``[n_cells, n, n]`` indexed ``[e, j, i]`` (i along x, j along y).
    """
    cells = np.asarray(cells, dtype=np.int64).reshape(-1, 3)
    lev, ix, iy = cells[:, 0], cells[:, 1], cells[:, 2]
    h = length / (2.0 ** lev)
    xl = x0 + ix * h
    yl = x0 + iy * h
    s = 0.5 * (np.asarray(xi, dtype=np.float64) + 1.0)
    X = xl[:, None, None] + h[:, None, None] * s[None, None, :]
    Y = yl[:, None, None] + h[:, None, None] * s[None, :, None]
    X = np.broadcast_to(X, (len(cells), len(s), len(s))).copy()
    Y = np.broadcast_to(Y, (len(cells), len(s), len(s))).copy()
    return X, Y


def nodal_state(ic, cells: Sequence, x0: float, length: float, xi: np.ndarray, **kw) -> np.ndarray:
    """Initial condition ``ic`` sampled at the nodes: array ``[n_cells, 4, n, n]``
    (conserved variable, then j along y, then i along x), C-contiguous float64."""
    X, Y = node_coordinates(cells, x0, length, xi)
    U = ic(X, Y, **kw)                       # [4, n_cells, n, n]
    return np.ascontiguousarray(np.moveaxis(U, 0, 1), dtype=np.float64)


def smooth_random_state(cells: Sequence, x0: float, length: float, xi: np.ndarray, seed: int = SEED,
                        n_modes: int = 3, amplitude: float = 0.05) -> np.ndarray:
    """Seeded smooth, positive state: background (rho, v1, v2, p) = (1, 0.3, -0.2, 1)
    plus a few random periodic Fourier modes of each primitive variable."""
    rng = np.random.default_rng(seed)
    X, Y = node_coordinates(cells, x0, length, xi)
    kx = 2.0 * math.pi / length
    prims = []
    for base in (1.0, 0.3, -0.2, 1.0):
        f = np.full_like(X, base)
        for _ in range(n_modes):
            a = amplitude * rng.uniform(-1.0, 1.0)
            mx, my = rng.integers(0, 3, size=2)
            ph = rng.uniform(0.0, 2.0 * math.pi)
            f = f + a * np.sin(kx * (mx * (X - x0) + my * (Y - x0)) + ph)
        prims.append(f)
    U = prim_to_cons(*prims)
    return np.ascontiguousarray(np.moveaxis(U, 0, 1), dtype=np.float64)
