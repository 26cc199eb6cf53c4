"""The fused small-instance steps against the tiled kernels (fused_small =
0) and the oracle: fused_small = 1, one CTA per instance of at most
HWENO_FUSED_MAX_POINTS points, and fused_small = 2, one thread-block cluster
per instance of at most HWENO_CLUSTER_MAX_POINTS points (one tile per CTA);
both run the wave speed, three stages and time update in one launch. The
stage code is shared; compiled into another kernel the compiler may fuse
a*b + c*d differently, so the paths agree to rounding."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2207_05258_gb300 import workloads as W
from _util import oracle_problem

pytestmark = pytest.mark.gpu
SIZES = [4, 5, 31, 123, 124, 125, 128, 248, 249, 400, 507, 508]
# the cluster step: up to eight 124-point tiles; ragged tile counts per batch
SIZES_CLUSTER = SIZES + [620, 871, 991, 992]
# instances of at most 448 points: the cluster step's latency form (28-point
# tiles, up to 16 per cluster, the work of a point over four warps)
SIZES_SPLIT = [4, 5, 27, 28, 29, 31, 56, 57, 124, 125, 248, 400, 447, 448]
MODES = {1: SIZES, 2: SIZES_CLUSTER, 3: SIZES_SPLIT}
FUSED = {1: 1, 2: 2, 3: 2}  # option value of each case


@pytest.fixture(scope="module")
def hw():
    from paper_2207_05258_gb300 import build
    build.build()
    from paper_2207_05258_gb300 import hweno
    return hweno


def _batch(eq, sizes, seed):
    rng = np.random.default_rng(seed)
    Us, Vs = [], []
    for k, n in enumerate(sizes):
        x = W.centers(0, 1, n)
        if eq == "euler":
            lo = x < rng.uniform(0.3, 0.7)
            rho = np.where(lo, 1.0, 0.125) + 0.1 * np.sin(2 * np.pi * x)
            u = 0.1 * np.cos(2 * np.pi * x)
            p = np.where(lo, 1.0, 0.1)
            Us.append(W.euler_conserved(rho, u, p, 1.4).ravel())
            Vs.append(np.zeros(3 * n))
        elif eq == "burgers":
            Us.append(0.3 + np.sin(2 * np.pi * x + rng.uniform(0, 6)))
            Vs.append(2 * np.pi * np.cos(2 * np.pi * x))
        else:
            Us.append(np.clip(0.5 + 0.45 * np.sin(2 * np.pi * x + rng.uniform(0, 6)), 0, 1))
            Vs.append(np.zeros(n))
    bc = "outflow" if eq == "euler" else "periodic"
    return W.Workload("fs", eq, 1, list(sizes), 1, 0.0, 1.0, 0.0, 1.0, 0.1,
                      (bc, bc, "periodic", "periodic"), np.concatenate(Us), np.concatenate(Vs))


def _steps(hw, w, K, t_end, precision="fp64", **opts):
    dt = torch.float64 if precision == "fp64" else torch.float32
    s = hw.Solver.from_workload(w, precision=precision, **opts)
    U = torch.from_numpy(w.U).to("cuda", dt)
    V = torch.from_numpy(w.V).to("cuda", dt)
    t = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
    used = []
    for _ in range(K):
        d = torch.empty(w.batch, dtype=torch.float64, device="cuda")
        s.step(U, V, None, t, t_end, d)
        used.append(d)
    s.sync_status()
    launches = s.launches_last_call
    act = s.active_instances()
    s.close()
    return U, V, t, torch.stack(used), act, launches


@pytest.mark.parametrize("mode", [1, 2, 3])
@pytest.mark.parametrize("eq", ["euler", "burgers", "buckley"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fused_matches_tiled(hw, eq, precision, mode):
    w = _batch(eq, MODES[mode], 3)
    K, t_end = 8, 0.01
    f = _steps(hw, w, K, t_end, precision, fused_small=FUSED[mode])
    g = _steps(hw, w, K, t_end, precision)
    assert f[5] == 1 and g[5] == 5          # one launch per step vs five
    ru = 1e-13 * K if precision == "fp64" else 1e-5 * K
    assert float((f[0] - g[0]).abs().max()) <= ru * float(g[0].abs().max())
    assert float((f[2] - g[2]).abs().max()) <= (1e-14 if precision == "fp64" else 1e-6) * K * 0.01
    assert torch.equal(f[3] > 0, g[3] > 0)  # the same instances step at the same steps
    assert f[4] == g[4]


@pytest.mark.parametrize("mode", [1, 2, 3])
@pytest.mark.parametrize("eq", ["euler", "burgers"])
def test_fused_against_the_oracle(hw, mode, eq):
    w = _batch(eq, MODES[mode], 4)
    m = 3 if eq == "euler" else 1
    U, V, t, used, act, _ = _steps(hw, w, 3, 1.0, fused_small=FUSED[mode])
    Ug = U.cpu().numpy()
    off = 0
    for k, n in enumerate(w.nx):
        Uk, Vk = w.instance(k)
        Uo, _, _, to, _ = O.run(oracle_problem(w, nx=n), Uk, Vk, None, 0.0, 1.0, max_steps=3)
        g = Ug[m * off:m * (off + n)].reshape(m, n)
        assert np.max(np.abs(g - Uo)) <= 1e-12 * np.max(np.abs(Uo)), (k, n)
        assert abs(float(t[k]) - to) <= 1e-14 * to
        off += n


@pytest.mark.parametrize("mode,n", [(1, 509), (2, 993)])
def test_larger_instances_use_the_tiled_kernels(hw, mode, n):
    w = _batch("burgers", [n, 40], 5)
    *_, launches = _steps(hw, w, 1, 1.0, fused_small=mode)
    assert launches == 5


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_finished_instances_do_not_move(hw, mode):
    """Instances whose time has reached t_end keep their state, report
    dt_used = 0 and are not counted active; the others step as in the tiled
    path."""
    w = _batch("euler", [40, 400, 700 if mode == 2 else 300], 6)
    s = hw.Solver.from_workload(w, fused_small=FUSED[mode])
    g = hw.Solver.from_workload(w)
    t_end = 0.05
    res = []
    for solver in (s, g):
        U = torch.from_numpy(w.U).cuda()
        V = torch.from_numpy(w.V).cuda()
        t = torch.tensor([0.0, t_end, 0.0], dtype=torch.float64, device="cuda")
        d = torch.empty(3, dtype=torch.float64, device="cuda")
        solver.step(U, V, None, t, t_end, d)
        solver.sync_status()
        res.append((U.cpu(), t.cpu(), d.cpu(), solver.active_instances()))
    (Uf, tf, df, af), (Ug, tg, dg, ag) = res
    off = 3 * 40
    n1 = 3 * 400
    assert torch.equal(Uf[off:off + n1], torch.from_numpy(w.U)[off:off + n1])
    assert float(df[1]) == 0.0 and float(tf[1]) == t_end
    assert float((Uf - Ug).abs().max()) <= 1e-13 * float(Ug.abs().max())
    assert torch.allclose(tf, tg, rtol=1e-14, atol=0) and af == ag == 2


@pytest.mark.parametrize("mode", [1, 2])
def test_burgers_n400_to_final_time(hw, mode):  # N = 400: mode 2 takes the latency form
    """Example 3.1 (Burgers N = 400, T = 1.5/pi, shock) through the
    fused paths against the oracle, shocked-run tolerance."""
    w = W.burgers1d_sine(400)
    s = hw.Solver.from_workload(w, fused_small=mode)
    U = torch.from_numpy(w.U).cuda()
    V = torch.from_numpy(w.V).cuda()
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    s.run(U, V, None, t, w.t_end)
    Uo, Vo, _, to, _ = O.run(oracle_problem(w), w.U, w.V, None, 0.0, w.t_end)
    assert float(t[0]) == to == w.t_end
    assert np.max(np.abs(U.cpu().numpy() - Uo.ravel())) <= 1e-8 * np.max(np.abs(Uo))
    assert s.launches_last_call >= 1


@pytest.mark.parametrize("mode", [2, 3])
def test_cluster_persistent_run_matches_the_steps(hw, mode):
    """hweno_run_persistent with fused_small = 2: the K steps as one launch of
    the cluster step give the bits of K single-step calls; instances that
    reach t_end on the way stop; the point-updates count the stepping ones."""
    w = _batch("euler", MODES[mode], 7)
    K, t_end = 6, 0.02
    a = hw.Solver.from_workload(w, fused_small=2)
    b = hw.Solver.from_workload(w, fused_small=2)
    U1, V1 = torch.from_numpy(w.U).cuda(), torch.from_numpy(w.V).cuda()
    U2, V2 = U1.clone(), V1.clone()
    t1 = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
    t2 = t1.clone()
    nx = torch.tensor(w.nx, dtype=torch.float64, device="cuda")
    pu_steps = 0.0
    for _ in range(K):
        d = torch.empty(w.batch, dtype=torch.float64, device="cuda")
        a.step(U1, V1, None, t1, t_end, d)
        pu_steps += float(((d > 0).double() * nx).sum())
    a.sync_status()
    pu = b.run_persistent(U2, V2, t2, t_end, K)
    assert b.launches_last_call == 1
    assert torch.equal(U1, U2) and torch.equal(V1, V2) and torch.equal(t1, t2)
    assert pu == pu_steps
    assert b.active_instances() == a.active_instances()
    assert 0 < a.active_instances() < w.batch  # some finished on the way
    a.close()
    b.close()


@pytest.mark.parametrize("mode", [1, 2, 3])
@pytest.mark.parametrize("eq,bc", [("euler", ("reflective", "inflow")),
                                   ("euler", ("inflow", "reflective")),
                                   ("burgers", ("reflective", "outflow")),
                                   ("buckley", ("inflow", "outflow"))])
def test_fused_boundaries_match_tiled(hw, mode, eq, bc):
    """Walls (mirrored ghosts) and imposed inflow states in the fused loads,
    against the tiled kernels."""
    import dataclasses
    w = _batch(eq, MODES[mode], 8)
    inflow = (1.0, 0.2, 2.6, 0.0) if eq == "euler" else (0.4, 0.0, 0.0, 0.0)
    w = dataclasses.replace(w, bc=(bc[0], bc[1], "periodic", "periodic"), inflow=inflow)
    K, t_end = 6, 0.01
    f = _steps(hw, w, K, t_end, "fp64", fused_small=FUSED[mode])
    g = _steps(hw, w, K, t_end, "fp64")
    assert f[5] == 1 and g[5] == 5
    assert float((f[0] - g[0]).abs().max()) <= 1e-13 * K * float(g[0].abs().max())
    assert float((f[1] - g[1]).abs().max()) <= 1e-12 * K * float(g[1].abs().max() + 1.0)
    assert torch.allclose(f[2], g[2], rtol=1e-14, atol=0)


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_fused_steps_in_a_cuda_graph(hw, mode):
    """hweno_run records the fused or cluster step into a CUDA graph (the
    first call on a fresh context, so the one-time set-up happens in the
    recording) and replays it: the bits of the same steps taken one by one."""
    w = _batch("burgers", MODES[mode], 9)
    K, t_end = 5, 0.02
    a = hw.Solver.from_workload(w, fused_small=FUSED[mode])
    b = hw.Solver.from_workload(w, fused_small=FUSED[mode])
    U1, V1 = torch.from_numpy(w.U).cuda(), torch.from_numpy(w.V).cuda()
    U2, V2 = U1.clone(), V1.clone()
    t1 = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
    t2 = t1.clone()
    for _ in range(K):
        a.step(U1, V1, None, t1, t_end)
    a.sync_status()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        steps, pu = b.run_graph(U2, V2, None, t2, t_end, max_steps=K, steps_per_launch=K)
    torch.cuda.synchronize()
    b.sync_status()
    assert steps == K and pu > 0
    assert torch.equal(U1, U2) and torch.equal(V1, V2) and torch.equal(t1, t2)
    a.close()
    b.close()
