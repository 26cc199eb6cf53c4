"""The persistent run (hweno_run_persistent: K steps of a ragged 1D batch in
one launch, work items taken in (step, stage, tile) order with per-instance
dependencies) against K plain hweno_step calls and against the oracle.

The stage code is the same, but compiled into another kernel the compiler
may contract an expression a*b + c*d into a different fused multiply-add, so
the two runs agree to rounding (FP64: a few ulps per step), not bit for bit;
point-update counts and the number of active instances must agree exactly,
also when instances reach t_end during the run. The oracle comparison uses
the 1D parity tolerances."""
import numpy as np
import pytest
import torch

from paper_2207_05258_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hw():
    from paper_2207_05258_gb300 import build
    build.build()
    from paper_2207_05258_gb300 import hweno
    return hweno


def _batch(eq, seed):
    if eq == "euler":
        return W.riemann_batch(count=96, seed=seed, sizes=(4, 31, 124, 125, 200, 400, 1600))
    rng = np.random.default_rng(seed)
    sizes = [int(n) for n in rng.choice([4, 60, 124, 125, 250, 800], 40)]
    Us, Vs = [], []
    for n in sizes:
        x = W.centers(-1, 1, n)
        if eq == "burgers":
            Us.append(0.3 + np.sin(np.pi * x + rng.uniform(0, 6)))
            Vs.append(np.pi * np.cos(np.pi * x))
        else:
            Us.append(np.clip(0.5 + 0.45 * np.sin(np.pi * x + rng.uniform(0, 6)), 0, 1))
            Vs.append(np.zeros(n))
    return W.Workload("pb", eq, 1, sizes, 1, -1.0, 1.0, 0.0, 1.0, 0.3,
                      ("periodic", "periodic", "periodic", "periodic"),
                      np.concatenate(Us), np.concatenate(Vs))


def _compare(hw, w, precision, variant, K, t_end):
    dt = torch.float64 if precision == "fp64" else torch.float32
    s = hw.Solver.from_workload(w, precision=precision, tile_variant=variant)
    U0 = torch.from_numpy(w.U).to("cuda", dt)
    V0 = torch.from_numpy(w.V).to("cuda", dt)
    # plain steps
    U1, V1 = U0.clone(), V0.clone()
    t1 = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
    nx = torch.tensor(w.nx, dtype=torch.float64, device="cuda")
    pu1 = 0.0
    for _ in range(K):
        d = torch.empty(w.batch, dtype=torch.float64, device="cuda")
        s.step(U1, V1, None, t1, t_end, d)
        pu1 += float(((d > 0).double() * nx).sum().item())
    s.sync_status()
    act1 = s.active_instances()
    # one persistent launch
    U2, V2 = U0.clone(), V0.clone()
    t2 = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
    pu2 = s.run_persistent(U2, V2, t2, t_end, K)
    act2 = s.active_instances()
    rt = 1e-14 * K if precision == "fp64" else 1e-6 * K
    ru = 1e-13 * K if precision == "fp64" else 1e-5 * K
    assert float(((t1 - t2).abs() / t1.abs().clamp_min(1e-300)).max()) <= rt
    su = float(U1.abs().max()) + 1e-300
    sv = float(V1.abs().max()) + 1e-300
    assert float((U1 - U2).abs().max()) <= ru * su
    assert float((V1 - V2).abs().max()) <= ru * 100 * sv
    assert pu1 == pu2, (pu1, pu2)
    assert act1 == act2
    s.close()
    return act2


@pytest.mark.parametrize("variant", range(5))
def test_euler_fp64_every_variant(hw, variant):
    w = _batch("euler", 7)
    _compare(hw, w, "fp64", variant, 6, 1.0)


@pytest.mark.parametrize("eq", ["euler", "burgers", "buckley"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_equations_and_precisions(hw, eq, precision):
    w = _batch(eq, 8)
    _compare(hw, w, precision, 0, 5, 1.0)


def test_instances_finish_during_the_run(hw):
    """t_end reached by the small instances after a few steps and by none of
    the large ones: the persistent run must stop stepping exactly the same
    instances at the same step."""
    w = _batch("euler", 9)
    act = _compare(hw, w, "fp64", 3, 12, 0.004)
    assert 0 < act < w.batch


def test_full_size_batch(hw):
    w = W.riemann_batch()
    _compare(hw, w, "fp64", 3, 3, w.t_end)


def test_against_the_oracle(hw):
    """Three persistent steps of a ragged Euler batch against the oracle's
    three steps, per instance, at the 1D one-step tolerances."""
    import oracle as O
    from _util import oracle_problem
    w = _batch("euler", 10)
    s = hw.Solver.from_workload(w)
    U = torch.from_numpy(w.U).cuda()
    V = torch.from_numpy(w.V).cuda()
    t = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
    s.run_persistent(U, V, t, 1.0, 3)
    Ug, tg = U.cpu().numpy(), t.cpu().numpy()
    off = 0
    for k, n in enumerate(w.nx):
        Uk, Vk = w.instance(k)
        Uo, _, _, to, _ = O.run(oracle_problem(w, nx=n), Uk, Vk, None, 0.0, 1.0, max_steps=3)
        g = Ug[3 * off:3 * (off + n)].reshape(3, n)
        assert np.max(np.abs(g - Uo)) <= 1e-12 * np.max(np.abs(Uo)), k
        assert abs(tg[k] - to) <= 1e-14 * to
        off += n


def test_a_wait_that_cannot_end_times_out_and_the_context_survives(hw):
    """Failure detection without a fault: the injected tile count makes
    instance 0's waits unsatisfiable; the bounded waits give up (about two
    seconds), the call reports ETIMEOUT, and afterwards plain and persistent
    steps of the same context work and agree with a fresh context."""
    import time
    w = _batch("euler", 12)
    s = hw.Solver.from_workload(w)
    U = torch.from_numpy(w.U).cuda()
    V = torch.from_numpy(w.V).cuda()
    t = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
    s.test_inject(1)
    t0 = time.perf_counter()
    with pytest.raises(hw.HwenoError) as err:
        s.run_persistent(U.clone(), V.clone(), t.clone(), 1.0, 2)
    assert err.value.code == hw.ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    # the context is usable again
    U1, V1, t1 = U.clone(), V.clone(), t.clone()
    s.run_persistent(U1, V1, t1, 1.0, 2)
    r = hw.Solver.from_workload(w)
    U2, V2, t2 = U.clone(), V.clone(), t.clone()
    r.run_persistent(U2, V2, t2, 1.0, 2)
    assert torch.equal(U1, U2) and torch.equal(t1, t2)
