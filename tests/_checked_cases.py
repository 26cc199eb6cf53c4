"""Cases run against the checked build of the library (device-side index
checks, NaN-filled stage scratch; see tests/test_gpu_checked_build.py).

Run as a script with HWENO_LIBRARY pointing at the checked library. Every
kernel family runs on small and ragged grids: the 1D stage kernels (right-hand
side and steps, every tile variant, Burgers and Euler, every boundary kind),
the persistent run, the cluster step, the 2D sweeps and the fused 2D stage,
the totals and the adjoint steps. Results are compared with the oracle where the plain build's
parity tests do, and the context's status must stay clean (a failed check
would come back as HWENO_EBOUNDS). Prints "CHECKED OK" at the end.
"""
import os
import sys

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path[:0] = [os.path.dirname(HERE), HERE]

import oracle as O  # noqa: E402
from paper_2207_05258_gb300 import hweno as hw  # noqa: E402
from paper_2207_05258_gb300 import workloads as W  # noqa: E402
from _util import oracle_problem  # noqa: E402

SIZES = [4, 5, 31, 123, 124, 125, 248, 249]


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def batch_1d(eq, bc, seed):
    rng = np.random.default_rng(seed)
    Us, Vs = [], []
    for n in SIZES:
        x = W.centers(0, 1, n)
        if eq == "burgers":
            Us.append(0.3 + np.sin(2 * np.pi * x + rng.uniform(0, 6)) + 0.1 * rng.standard_normal(n))
            Vs.append(rng.standard_normal(n))
        else:
            rho = 1 + 0.3 * np.sin(2 * np.pi * x + rng.uniform(0, 6)) + 0.05 * rng.uniform(-1, 1, n)
            u = 0.2 * np.cos(2 * np.pi * x)
            p = 1 + 0.1 * rng.uniform(-1, 1, n)
            Us.append(W.euler_conserved(rho, u, p, 1.4).ravel())
            Vs.append(rng.standard_normal(3 * n))
    return W.Workload("chk", eq, 1, SIZES, 1, 0.0, 1.0, 0.0, 1.0, 0.3,
                      (bc, bc, "periodic", "periodic"), np.concatenate(Us), np.concatenate(Vs),
                      inflow=(0.7, 0, 0, 0) if eq == "burgers" else (1.0, 0.2, 2.6, 0.0))


def split(w, flat):
    out, off = [], 0
    for n in w.nx:
        out.append(flat[off:off + w.m * n].reshape(w.m, n))
        off += w.m * n
    return out


def check_1d(w, variant, fused=0):
    s = hw.Solver.from_workload(w, tile_variant=variant, fused_small=fused)
    U, V = dev(w.U), dev(w.V)
    r = s.rhs(U, V)
    t = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
    dt = torch.zeros_like(t)
    for _ in range(2):
        s.step(U, V, None, t, w.t_end, dt)
    s.sync_status()
    GU, L1 = split(w, U.cpu().numpy()), split(w, r["L1"].cpu().numpy())
    for k, n in enumerate(w.nx):
        Uk, Vk = w.instance(k)
        P = oracle_problem(w, nx=n)
        ro = O.rhs(P, Uk, Vk)
        scale = np.max(np.abs(ro["L1"])) + 1.0
        assert np.max(np.abs(L1[k] - ro["L1"])) <= 1e-10 * scale, ("rhs", w.equation, n)
        Uo = O.run(P, Uk, Vk, None, 0.0, w.t_end, max_steps=2)[0]
        assert np.max(np.abs(GU[k] - Uo)) <= 1e-11 * np.max(np.abs(Uo)), ("step", w.equation, n)
    # the adjoint of one step (Burgers / Euler FP64)
    if w.bc[0] != "inflow":
        lU, lV = torch.ones_like(U), torch.ones_like(V)
        t0 = torch.zeros_like(t)
        s.adjoint_step(dev(w.U), dev(w.V), None, dt, lU, lV, t=t0)
        s.sync_status()
        assert torch.isfinite(lU).all() and torch.isfinite(lV).all()
    tot = s.totals(U)
    s.sync_status()
    assert torch.isfinite(tot).all()
    s.close()


def main():
    for eq in ("burgers", "euler"):
        for bc in ("periodic", "outflow", "reflective", "inflow"):
            w = batch_1d(eq, bc, 7)
            for v in range(hw.TILE_VARIANTS):
                check_1d(w, v)
    # persistent run and the cluster step (small instances)
    full = W.riemann_batch(count=12, seed=4)
    for fused in (0, 2):
        sub = [k for k in range(12) if full.nx[k] <= 800][:4] if fused else list(range(12))
        Us, Vs = zip(*(full.instance(k) for k in sub))
        w = W.Workload("p", "euler", 1, [full.nx[k] for k in sub], 1, 0.0, 1.0, 0.0, 1.0, 0.15,
                       full.bc, np.concatenate([u.ravel() for u in Us]),
                       np.concatenate([v.ravel() for v in Vs]))
        s = hw.Solver.from_workload(w, fused_small=fused)
        U, V = dev(w.U), dev(w.V)
        t = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
        s.run_persistent(U, V, t, w.t_end, 3)
        for k, n in enumerate(w.nx):
            Uk, Vk = w.instance(k)
            Uo = O.run(oracle_problem(w, nx=n), Uk, Vk, None, 0.0, w.t_end, max_steps=3)[0]
            g = split(w, U.cpu().numpy())[k]
            assert np.max(np.abs(g - Uo)) <= 1e-11 * np.max(np.abs(Uo)), ("persistent", fused, n)
        s.close()
    # 2D: smooth periodic, walls and inflow, the double Mach boundaries; rhs,
    # two steps (split and fused stage forms) and one adjoint step
    cases = [W.euler2d_smooth(24, ny=13, t_end=1.0), W.double_mach(40, 12, t_end=1.0),
             W.burgers2d_sine(20)]
    for w, fused in [(w, f) for w in cases for f in (0, 1)]:
        s = hw.Solver.from_workload(w, fused_2d=fused)
        U, V, Wd = dev(w.U), dev(w.V), dev(w.W)
        s.rhs(U, V, Wd)
        t = torch.zeros(1, dtype=torch.float64, device="cuda")
        dt = torch.zeros_like(t)
        for _ in range(2):
            s.step(U, V, Wd, t, w.t_end, dt)
        s.sync_status()
        Uo = O.run(oracle_problem(w), w.U, w.V, w.W, 0.0, w.t_end, max_steps=2)[0]
        g = U.cpu().numpy().reshape(Uo.shape)
        assert np.max(np.abs(g - Uo)) <= 1e-11 * np.max(np.abs(Uo)), ("2d", w.name, fused)
        if w.bc[0] == "periodic":
            lam = [torch.ones_like(U), torch.ones_like(V), torch.ones_like(Wd)]
            s.adjoint_step(dev(w.U), dev(w.V), dev(w.W), dt, *lam, t=torch.zeros_like(t))
            s.sync_status()
            assert all(torch.isfinite(x).all() for x in lam)
        s.close()
        # FP32 (packed pairs, asynchronous tile copies in the y-sweep)
        s = hw.Solver.from_workload(w, precision="fp32", fused_2d=fused)
        f32 = lambda x: dev(x).float()
        U, V, Wd = f32(w.U), f32(w.V), f32(w.W)
        s.rhs(U, V, Wd)
        t = torch.zeros(1, dtype=torch.float64, device="cuda")
        for _ in range(2):
            s.step(U, V, Wd, t, w.t_end)
        s.sync_status()
        g = U.double().cpu().numpy().reshape(Uo.shape)
        assert np.max(np.abs(g - Uo)) <= 1e-4 * np.max(np.abs(Uo)), ("2d fp32", w.name, fused)
        s.close()
    # the checks are live: the self-test latches HWENO_EBOUNDS, and the
    # context works afterwards
    w = batch_1d("burgers", "periodic", 3)
    s = hw.Solver.from_workload(w)
    s.test_inject(2)
    try:
        s.sync_status()
        raise AssertionError("the self-test did not latch HWENO_EBOUNDS")
    except hw.HwenoError as e:
        assert e.code == hw.EBOUNDS, e
    check_1d(w, 0)
    print("CHECKED OK")


if __name__ == "__main__":
    main()
