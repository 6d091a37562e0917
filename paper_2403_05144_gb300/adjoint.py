"""Discrete adjoint of the P-ERK step for PyTorch users.

``PerkStep`` is a ``torch.autograd.Function`` around ``perk_step`` /
``perk_step_vjp``: its backward is the library's reverse sweep of the step
(Jacobian transposes of the partitioned RHS and of the stage combinations).
``gradient`` differentiates a functional of the end state over many steps on a
frozen mesh with step checkpointing: the state is stored every
``checkpoint_every`` steps and each window's steps are recomputed from its
checkpoint during the reverse sweep, keeping their stages, so memory holds one
window of states and stages.
"""

from __future__ import annotations

from typing import Callable

import torch

from . import PerkSolver


class PerkStep(torch.autograd.Function):
    """U_{n+1} = P-ERK step of U_n (out of place), differentiable in U_n."""

    @staticmethod
    def forward(ctx, U, solver: PerkSolver, dt: float):
        ctx.solver = solver
        ctx.dt = dt
        ctx.save_for_backward(U)
        Un = U.detach().clone()
        solver.step(Un, dt)
        return Un

    @staticmethod
    def backward(ctx, grad):
        (U,) = ctx.saved_tensors
        lam = ctx.solver.step_vjp(U.detach().contiguous(), ctx.dt, grad.contiguous())
        return lam, None, None


def kinetic_energy(U: torch.Tensor, h: torch.Tensor, w: torch.Tensor) -> torch.Tensor:
    """J = (1/2) sum over cells and nodes of (h_e/2)^2 w_i w_j |rho v|^2 / rho (the LGL quadrature)."""
    rho, m1, m2 = U[:, 0], U[:, 1], U[:, 2]
    W = (0.5 * h)[:, None, None] ** 2 * torch.outer(w, w)[None]
    return 0.5 * torch.sum(W * (m1 * m1 + m2 * m2) / rho)


def gradient(solver: PerkSolver, U0: torch.Tensor, dt: float, n_steps: int,
             functional: Callable[[torch.Tensor], torch.Tensor], checkpoint_every: int = 20,
             store_stages: bool = True):
    """(J(U_N), dJ/dU_0) for N = n_steps P-ERK steps from U0 on the solver's (frozen) mesh.

    With ``store_stages`` the recomputation of a window keeps every step's stages
    (checkpoint_every x S states) and the reverse sweep reads them; otherwise each
    reverse step recomputes its own stages."""
    checkpoints = {}
    U = U0.detach().clone()
    for n in range(n_steps):
        if n % checkpoint_every == 0:
            checkpoints[n] = U.clone()
        solver.step(U, dt)
    UN = U.detach().requires_grad_(True)
    J = functional(UN)
    (lam,) = torch.autograd.grad(J, UN)
    lam = lam.contiguous()
    lam_next = torch.empty_like(lam)
    starts = sorted(checkpoints)
    buf = None
    if store_stages:
        buf = torch.empty((min(checkpoint_every, n_steps), solver.S) + tuple(U0.shape), dtype=U0.dtype,
                          device=U0.device)
    for w_start in reversed(starts):
        w_end = min(w_start + checkpoint_every, n_steps)
        Uw = checkpoints[w_start].clone()
        states = []
        for k in range(w_end - w_start):
            states.append(Uw.clone())
            if store_stages:
                solver.step_store(Uw, dt, stages=buf[k])
            elif k < w_end - w_start - 1:
                solver.step(Uw, dt)
        for k in reversed(range(len(states))):
            solver.step_vjp(states[k], dt, lam, out=lam_next, stages=buf[k] if store_stages else None)
            lam, lam_next = lam_next, lam
    solver.check()
    return J.detach(), lam
