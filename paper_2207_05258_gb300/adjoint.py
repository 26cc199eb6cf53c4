"""Gradients of a final-time functional through a run of hweno_step: a
torch.autograd.Function whose backward is the library's discrete adjoint
(hweno_adjoint_step), with checkpoints every k steps and recomputation of the
states inside each segment.

The derivative is that of the discrete scheme with the per-stage wave speeds
and the time steps frozen (constants of the run) and the |.| branches of the
smoothness differences taken at the forward states; the nonlinear weights,
the characteristic eigenvectors and the limiter are differentiated.
"""
from __future__ import annotations

import torch


class RunToTime(torch.autograd.Function):
    """(U(T), V(T)[, W(T)]) = run(U0, V0[, W0]) from t = 0 to t_end with an
    FP64 `solver` (W0 None in 1D)."""

    @staticmethod
    def forward(ctx, U0, V0, W0, solver, t_end, checkpoint_every, max_steps, check_every):
        two = W0 is not None
        U, V = U0.detach().clone(), V0.detach().clone()
        W = W0.detach().clone() if two else None
        t = torch.zeros(solver.batch, dtype=torch.float64, device=U.device)
        checkpoints, dts, ts = [], [], []
        k = 0
        while k < max_steps:
            if k % checkpoint_every == 0:
                checkpoints.append((k, U.clone(), V.clone(), W.clone() if two else None,
                                    t.clone()))
            ts.append(t.clone())
            dt = torch.empty(solver.batch, dtype=torch.float64, device=U.device)
            solver.step(U, V, W, t, t_end, dt)
            dts.append(dt)
            k += 1
            if k % check_every == 0 and solver.active_instances() == 0:
                break
        solver.sync_status()
        ctx.solver, ctx.t_end, ctx.checkpoints = solver, t_end, checkpoints
        ctx.dts, ctx.ts, ctx.steps, ctx.two = dts, ts, k, two
        return (U, V, W) if two else (U, V)

    @staticmethod
    def backward(ctx, *grads):
        solver, two = ctx.solver, ctx.two
        lam = [g.detach().clone().contiguous() for g in grads]
        bounds = [c[0] for c in ctx.checkpoints] + [ctx.steps]
        seg_len = max(bounds[i + 1] - bounds[i] for i in range(len(bounds) - 1))
        records = [solver.new_record(lam[0].device) for _ in range(seg_len)]
        for seg in range(len(ctx.checkpoints) - 1, -1, -1):
            k0, U, V, W, t = ctx.checkpoints[seg]
            k1 = bounds[seg + 1]
            U, V, t = U.clone(), V.clone(), t.clone()
            W = W.clone() if two else None
            states = []
            # replay the segment, keeping each step's input and its stage
            # states (a step record), so that the adjoint steps replay nothing
            for k in range(k0, k1):
                rec = records[k - k0]
                states.append((U.clone(), V.clone(), W.clone() if two else None))
                solver.step_record(U, V, W, t, ctx.t_end, rec)
            for k in range(k1 - 1, k0 - 1, -1):
                Uk, Vk, Wk = states[k - k0]
                solver.adjoint_step(Uk, Vk, Wk, ctx.dts[k], lam[0], lam[1],
                                    lam[2] if two else None, t=ctx.ts[k],
                                    record=records[k - k0])
        solver.sync_status()
        return (lam[0], lam[1], lam[2] if two else None, None, None, None, None, None)


def run_to_time(U0, V0, solver, t_end, checkpoint_every=20, max_steps=1 << 30, check_every=16,
                W0=None):
    """Differentiable run of an FP64 `solver` from (U0, V0[, W0]) at t = 0 to
    t_end; returns (U(T), V(T)[, W(T)]). Memory: one state per checkpoint
    plus, during the backward pass, one segment of states and step records
    (the stage states of each step: two more states per step)."""
    return RunToTime.apply(U0, V0, W0, solver, t_end, checkpoint_every, max_steps, check_every)
