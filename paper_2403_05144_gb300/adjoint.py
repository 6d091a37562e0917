"""Discrete adjoint of the P-ERK step for PyTorch users.

``PerkStep`` is a ``torch.autograd.Function`` around ``perk_step`` /
``perk_step_vjp``: its backward is the library's reverse sweep of the step
(Jacobian transposes of the partitioned RHS and of the stage combinations).
``gradient`` differentiates a functional of the end state over many steps on a
frozen mesh with step checkpointing: the state is stored every
``checkpoint_every`` steps; the windows whose stages fit in a device-memory
budget (the last ones, which the reverse sweep meets first) keep their states
and stages from the forward pass itself, and every other window's steps are
recomputed from its checkpoint during the reverse sweep, keeping their stages
in one reused buffer.
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
             store_stages: bool = True, memory_budget: int | None = None):
    """(J(U_N), dJ/dU_0) for N = n_steps P-ERK steps from U0 on the solver's (frozen) mesh.

    With ``store_stages`` the reverse sweep reads every step's stages (S states per
    step): the last windows of ``checkpoint_every`` steps keep theirs from the forward
    pass, as many as fit in ``memory_budget`` bytes (default: half the free device
    memory), and the others recompute them from their checkpoint into one reused
    buffer.  Without it each reverse step recomputes its own stages.  Returns the
    functional and the gradient; ``gradient.last_stats`` holds the windows kept."""
    n_windows = (n_steps + checkpoint_every - 1) // checkpoint_every
    state_bytes = U0.numel() * U0.element_size()
    window_bytes = checkpoint_every * (solver.S + 1) * state_bytes
    kept = 0
    if store_stages:
        if memory_budget is None:
            free, _ = torch.cuda.mem_get_info(U0.device)
            memory_budget = free // 2
        kept = int(min(n_windows, max(0, memory_budget) // window_bytes))
    first_kept = n_windows - kept                # windows first_kept.. keep their forward stages
    checkpoints, stored = {}, {}
    U = U0.detach().clone()
    for w in range(n_windows):
        w_start, w_end = w * checkpoint_every, min((w + 1) * checkpoint_every, n_steps)
        if w < first_kept:
            checkpoints[w_start] = U.clone()
            for _ in range(w_end - w_start):
                solver.step(U, dt)
        else:
            K = torch.empty((w_end - w_start, solver.S) + tuple(U0.shape), dtype=U0.dtype, device=U0.device)
            states = []
            for k in range(w_end - w_start):
                states.append(U.clone())
                solver.step_store(U, dt, stages=K[k])
            stored[w_start] = (states, K)
    UN = U.detach().requires_grad_(True)
    J = functional(UN)
    (lam,) = torch.autograd.grad(J, UN)
    lam = lam.contiguous()
    lam_next = torch.empty_like(lam)
    buf = None
    if store_stages and first_kept > 0:
        buf = torch.empty((min(checkpoint_every, n_steps), solver.S) + tuple(U0.shape), dtype=U0.dtype,
                          device=U0.device)
    for w in reversed(range(n_windows)):
        w_start, w_end = w * checkpoint_every, min((w + 1) * checkpoint_every, n_steps)
        if w_start in stored:
            states, K = stored.pop(w_start)
        else:
            Uw = checkpoints[w_start].clone()
            states, K = [], buf
            for k in range(w_end - w_start):
                states.append(Uw.clone())
                if store_stages:
                    solver.step_store(Uw, dt, stages=buf[k])
                elif k < w_end - w_start - 1:
                    solver.step(Uw, dt)
        for k in reversed(range(len(states))):
            solver.step_vjp(states[k], dt, lam, out=lam_next, stages=K[k] if store_stages else None)
            lam, lam_next = lam_next, lam
        del states, K
    solver.check()
    gradient.last_stats = {"windows": n_windows, "windows_kept_from_forward": kept,
                           "windows_recomputed": n_windows - kept, "window_bytes": window_bytes}
    return J.detach(), lam
