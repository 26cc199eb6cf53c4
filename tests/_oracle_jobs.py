"""Oracle runs of the full-size parity tests (tests/test_gpu_full_size.py).

Each function rebuilds its seeded input from paper_2207_05258_gb300.workloads
and runs the CPU oracle on it; the test submits them to a pool of spawned
worker processes so that they run on the host cores while the GPU works.
Nothing here touches a GPU.
"""
import numpy as np

import oracle as O
from paper_2207_05258_gb300 import workloads as W
from _util import oracle_problem

RIEMANN_SEED = 20220711  # the seeded 2048-instance batch of the benchmark


def riemann_instance(k):
    """Instance k of the 2048-instance Riemann batch, run to its final time
    (0.15): (U, V, t, steps)."""
    full = W.riemann_batch(count=2048, seed=RIEMANN_SEED)
    U, V = full.instance(k)
    U2, V2, _, t, n = O.run(oracle_problem(full, nx=full.nx[k]), U, V, None, 0.0, full.t_end)
    return U2, V2, t, n


def euler2d_smooth_steps(n, steps):
    """The 2D smooth periodic Euler workload (CFL time steps) on n x n after
    `steps` steps: (U, V, W, t)."""
    w = W.euler2d_smooth(n, dt_mode="cfl")
    U, V, Wd, t, _ = O.run(oracle_problem(w), w.U, w.V, w.W, 0.0, w.t_end, max_steps=steps)
    return U, V, Wd, t


def double_mach_steps(nx, ny, steps):
    """The double-Mach workload on nx x ny after `steps` steps: (U, V, W, t)."""
    w = W.double_mach(nx, ny)
    U, V, Wd, t, _ = O.run(oracle_problem(w), w.U, w.V, w.W, 0.0, w.t_end, max_steps=steps)
    return U, V, Wd, t


def adjoint_direction(n, seed, j):
    """Direction j of the 2D adjoint check: a seeded smooth perturbation of the
    initial density alone, with its exact x and y derivatives."""
    rng = W.SplitMix64(seed)
    for _ in range(j + 1):
        f, fx, fy = W.fourier_2d(rng, n, n, 0.0, 2.0, 1e-2)
    z = np.zeros(3 * n * n)
    return [np.concatenate([g.ravel(), z]) for g in (f, fx, fy)]


def euler2d_adjoint_tangent(n, wseed, dseed, j, steps):
    """Forward-mode (dual-number) derivative of J = sum(rho(T)^2) dx dy after
    `steps` fixed steps of the 2D Euler adjoint workload, along direction j:
    returns dJ."""
    w = W.euler2d_adjoint(n, seed=wseed)
    P = oracle_problem(w, dt_mode=2, dt_fixed=w.meta["dt"])
    d = adjoint_direction(n, dseed, j)
    out = O.run_tangent(P, w.U, w.V, w.W, d[0], d[1], d[2], 0.0, 1e30, max_steps=steps)
    cell = ((w.x1 - w.x0) / n) ** 2
    rho, drho = out[0][0], out[3][0]
    return float(np.sum(2.0 * rho * drho) * cell)
