"""Parity with the oracle at the benchmark workloads' full sizes, in the
launch configurations the benchmark times.

* 1D Euler Riemann batch (2048 seeded instances, N in {200 .. 3200}): the
  whole batch runs to t = 0.15 through persistent launches (the FP64
  headline path); the first instances of 1600 and 3200 points are compared
  with the oracle's run to the same time (shocked: relative L-inf <= 1e-8 on
  U and V; t bit-close).
* 2D smooth periodic Euler (Example 3.9) on 256^2, 10 CFL steps: the whole
  grid against the oracle (smooth: <= 1e-10).
* Double Mach reflection (Example 3.11) on 3840 x 960, one step: the whole
  grid against the oracle (one step: <= 1e-13 on U, 1e-11 on the
  derivatives, as for the other one-step 2D checks).
* 2D Euler adjoint workload on 512^2, 5 fixed steps with a checkpoint every
  2 steps: <grad J, d> of the checkpointed autograd Function against the
  oracle's dual-number tangent of J = sum(rho(T)^2) dx dy along 2 seeded
  directions (<= 1e-10 relative).

The oracle runs go to a pool of spawned processes at module start, so they
run on the host cores while the GPU works.
"""
import multiprocessing as mp

import numpy as np
import pytest
import torch

from paper_2207_05258_gb300 import workloads as W
import _oracle_jobs as J
from _util import max_err

pytestmark = pytest.mark.gpu

RIEMANN_PICK = (1, 7)  # the first 3200- and 1600-point instances of the seeded batch
ADJ_N, ADJ_STEPS, ADJ_WSEED, ADJ_DSEED = 512, 5, 7, 4321


@pytest.fixture(scope="module")
def hw():
    from paper_2207_05258_gb300 import build
    build.build()
    from paper_2207_05258_gb300 import hweno
    return hweno


@pytest.fixture(scope="module")
def jobs():
    """Submit every oracle run of this module at once (spawned workers)."""
    pool = mp.get_context("spawn").Pool(processes=6)
    res = {
        ("riemann", k): pool.apply_async(J.riemann_instance, (k,)) for k in RIEMANN_PICK}
    res["smooth"] = pool.apply_async(J.euler2d_smooth_steps, (256, 10))
    res["dmr"] = pool.apply_async(J.double_mach_steps, (3840, 960, 1))
    for j in range(2):
        res[("adj", j)] = pool.apply_async(J.euler2d_adjoint_tangent,
                                           (ADJ_N, ADJ_WSEED, ADJ_DSEED, j, ADJ_STEPS))
    pool.close()
    yield res
    pool.terminate()
    pool.join()


def test_riemann_batch_to_final_time_at_full_size(hw, jobs):
    w = W.riemann_batch(count=2048, seed=J.RIEMANN_SEED)
    assert [w.nx[k] for k in RIEMANN_PICK] == [3200, 1600]
    s = hw.Solver.from_workload(w)
    U = torch.from_numpy(w.U.copy()).cuda()
    V = torch.from_numpy(w.V.copy()).cuda()
    t = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
    s.autotune(U, V, None, t, w.t_end)
    for _ in range(40):  # 40 x 256 steps is more than any instance needs
        s.run_persistent(U, V, t, w.t_end, 256)
        if s.active_instances() == 0:
            break
    assert s.active_instances() == 0
    off = w.offsets
    GU, GV, gt = U.cpu().numpy(), V.cpu().numpy(), t.cpu().numpy()
    for k in RIEMANN_PICK:
        U2, V2, t2, steps = jobs[("riemann", k)].get(timeout=600)
        n = w.nx[k]
        sl = slice(3 * int(off[k]), 3 * (int(off[k]) + n))
        eu = max_err(GU[sl].reshape(3, n), U2) / np.max(np.abs(U2))
        ev = max_err(GV[sl].reshape(3, n), V2) / np.max(np.abs(V2))
        print("riemann instance %d (N = %d, %d steps): rel Linf U %.2e V %.2e"
              % (k, n, steps, eu, ev))
        assert eu <= 1e-8 and ev <= 1e-8, (k, eu, ev)
        assert gt[k] == w.t_end and t2 == w.t_end


def _run2d(hw, w, steps):
    s = hw.Solver.from_workload(w)
    U = torch.from_numpy(w.U.copy()).cuda()
    V = torch.from_numpy(w.V.copy()).cuda()
    Wd = torch.from_numpy(w.W.copy()).cuda()
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(steps):
        s.step(U, V, Wd, t, w.t_end)
    s.sync_status()
    return U.cpu().numpy(), V.cpu().numpy(), Wd.cpu().numpy(), float(t.item())


def _compare2d(w, g, o, rtol_u, rtol_vw):
    shp = (w.m, w.ny, w.nx[0])
    e = [max_err(g[i].reshape(shp), o[i]) / np.max(np.abs(o[i])) for i in range(3)]
    print("%s %dx%d: rel Linf U %.2e V %.2e W %.2e" % ((w.name, w.nx[0], w.ny) + tuple(e)))
    assert e[0] <= rtol_u and e[1] <= rtol_vw and e[2] <= rtol_vw, e
    assert abs(g[3] - o[3]) <= 1e-14 * o[3]


def test_smooth_2d_euler_256_ten_steps_whole_grid(hw, jobs):
    w = W.euler2d_smooth(256, dt_mode="cfl")
    g = _run2d(hw, w, 10)
    _compare2d(w, g, jobs["smooth"].get(timeout=600), 1e-10, 1e-10)


def test_double_mach_3840x960_one_step_whole_grid(hw, jobs):
    w = W.double_mach(3840, 960)
    g = _run2d(hw, w, 1)
    _compare2d(w, g, jobs["dmr"].get(timeout=900), 1e-13, 1e-11)


def test_adjoint_512_checkpointed_against_dual_numbers(hw, jobs):
    from paper_2207_05258_gb300.adjoint import run_to_time
    n = ADJ_N
    w = W.euler2d_adjoint(n, seed=ADJ_WSEED)
    s = hw.Solver.from_workload(w, dt_mode=2, dt_fixed=w.meta["dt"])
    cuda = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    U0 = cuda(w.U).requires_grad_(True)
    V0 = cuda(w.V).requires_grad_(True)
    W0 = cuda(w.W).requires_grad_(True)
    UT, _, _ = run_to_time(U0, V0, s, 1e30, 2, max_steps=ADJ_STEPS, W0=W0)
    cell = ((w.x1 - w.x0) / n) ** 2
    Jv = (UT[:n * n] ** 2).sum() * cell
    Jv.backward()
    g = [U0.grad.cpu().numpy(), V0.grad.cpu().numpy(), W0.grad.cpu().numpy()]
    for j in range(2):
        d = J.adjoint_direction(n, ADJ_DSEED, j)
        adj = float(sum(np.dot(gi, di) for gi, di in zip(g, d)))
        dJ = jobs[("adj", j)].get(timeout=900)
        cs = np.sqrt(sum(np.dot(gi, gi) for gi in g) * sum(np.dot(di, di) for di in d))
        print("adjoint 512^2 direction %d: <grad J, d> %.15e, dual %.15e, rel %.2e (|dJ| / CS "
              "scale %.2e)" % (j, adj, dJ, abs(adj - dJ) / abs(dJ), abs(dJ) / cs))
        assert abs(adj - dJ) <= 1e-10 * abs(dJ), (j, adj, dJ)
