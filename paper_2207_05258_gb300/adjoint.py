"""Gradients of a final-time functional through a run of hweno_step: a
torch.autograd.Function whose backward is the library's discrete adjoint
(hweno_adjoint_step), with checkpoints every k steps and recomputation of the
states inside each segment.

The derivative is that of the discrete scheme with the per-stage wave speed
alpha and the time steps frozen (constants of the run) and the |.| branches
of the smoothness differences taken at the forward states; the nonlinear
weights and the limiter are differentiated.
"""
from __future__ import annotations

import torch

from . import hweno


class RunToTime(torch.autograd.Function):
    """(U(T), V(T)) = run(U0, V0) to t_end with `solver` (1D, FP64)."""

    @staticmethod
    def forward(ctx, U0, V0, solver, t_end, checkpoint_every=20, max_steps=1 << 30,
                check_every=16):
        U, V = U0.detach().clone(), V0.detach().clone()
        t = torch.zeros(solver.batch, dtype=torch.float64, device=U.device)
        checkpoints, dts = [], []
        k = 0
        while k < max_steps:
            if k % checkpoint_every == 0:
                checkpoints.append((k, U.clone(), V.clone(), t.clone()))
            dt = torch.empty(solver.batch, dtype=torch.float64, device=U.device)
            solver.step(U, V, None, t, t_end, dt)
            dts.append(dt)
            k += 1
            if k % check_every == 0 and solver.active_instances() == 0:
                break
        solver.sync_status()
        ctx.solver, ctx.t_end, ctx.checkpoints, ctx.dts = solver, t_end, checkpoints, dts
        ctx.steps = k
        return U, V

    @staticmethod
    def backward(ctx, gU, gV):
        solver, dts = ctx.solver, ctx.dts
        lamU = gU.detach().clone().contiguous()
        lamV = gV.detach().clone().contiguous() if gV is not None else torch.zeros_like(lamU)
        bounds = [c[0] for c in ctx.checkpoints] + [ctx.steps]
        for seg in range(len(ctx.checkpoints) - 1, -1, -1):
            k0, U, V, t = ctx.checkpoints[seg]
            k1 = bounds[seg + 1]
            U, V, t = U.clone(), V.clone(), t.clone()
            states = []
            for k in range(k0, k1):  # replay the segment, keeping each step's input
                states.append((U.clone(), V.clone()))
                solver.step(U, V, None, t, ctx.t_end)
            for k in range(k1 - 1, k0 - 1, -1):
                Uk, Vk = states[k - k0]
                solver.adjoint_step(Uk, Vk, None, dts[k], lamU, lamV)
        solver.sync_status()
        return lamU, lamV, None, None, None, None, None


def run_to_time(U0, V0, solver, t_end, checkpoint_every=20, max_steps=1 << 30, check_every=16):
    """Differentiable run of a 1D Burgers FP64 `solver` from (U0, V0) at t = 0
    to t_end; returns (U(T), V(T)). Memory: one state per checkpoint plus one
    segment of states during the backward pass."""
    return RunToTime.apply(U0, V0, solver, t_end, checkpoint_every, max_steps, check_every)
