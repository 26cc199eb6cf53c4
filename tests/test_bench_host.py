"""Host-side pieces of bench.py: the algorithmic flop constants equal the
oracle's operation count, and the multi-rank reduction (max time, summed
work) over world_size 2 with the gloo backend on CPU."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import oracle as O
from paper_2207_05258_gb300 import workloads as W
from _util import oracle_problem


@pytest.mark.parametrize("key,make", [
    (("euler", 1), lambda: W.euler1d_smooth(1000, dt_mode="cfl")),
    (("burgers", 1), lambda: W.burgers1d_sine(1000)),
    (("buckley", 1), lambda: W.buckley_leverett(1000)),
    (("euler", 2), lambda: W.euler2d_smooth(64)),
    (("burgers", 2), lambda: W.burgers2d_sine(64)),
])
def test_flop_constants_match_oracle_count(key, make):
    w = make()
    n = O.flops_per_point_step(oracle_problem(w), w.U, w.V, w.W)
    assert abs(n - bench.ALGO_FLOPS_PER_POINT_STEP[key]) <= 1e-3 * n


@pytest.mark.parametrize("key,make", [
    (("euler", 2), lambda: W.euler2d_adjoint(64)),
    (("burgers", 1), lambda: W.burgers_adjoint_batch(count=1, n=800)),
])
def test_adjoint_flop_constants_match_oracle_tangent_count(key, make):
    """The adjoint step's algorithmic flops are the op count of the oracle's
    dual-number step (values and tangents) on the adjoint workloads."""
    w = make()
    kw = dict(dt_mode=2, dt_fixed=w.meta["dt"]) if w.dim == 2 else {}
    rng = np.random.default_rng(0)
    d = [rng.standard_normal(w.U.size) for _ in range(3 if w.dim == 2 else 2)]
    n = O.tangent_flops_per_point_step(oracle_problem(w, nx=w.nx[0], **kw), w.U, w.V, w.W, *d)
    assert abs(n - bench.ALGO_ADJOINT_FLOPS_PER_POINT_STEP[key]) <= 1e-3 * n


def test_tangent_count_is_value_count_plus_tangent_work():
    """The dual-number count includes the value arithmetic: it exceeds the
    plain step's count, by less than the four operations per multiply and
    divide that a tangent can add."""
    w = W.euler1d_smooth(200, dt_mode="cfl")
    P = oracle_problem(w)
    f = O.flops_per_point_step(P, w.U, w.V)
    tf = O.tangent_flops_per_point_step(P, w.U, w.V, None, np.ones_like(w.U), np.ones_like(w.V))
    assert 2.0 * f < tf < 5.0 * f


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, pu = bench.reduce_over_ranks(10.0 + rank, 100.0 * (rank + 1), "cpu")
    q.put((rank, ms, pu, bench.rank_seed(rank)))
    dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [11.0, 11.0]
    assert [o[2] for o in out] == [300.0, 300.0]
    assert out[0][3] != out[1][3]


def test_cpu_baseline_all_cores_on_a_small_sample():
    """The all-core oracle baseline (spawned processes) runs on CPU and
    reports the processes it used."""
    import bench
    from paper_2207_05258_gb300 import workloads as W
    w = W.riemann_batch(count=6, seed=3, sizes=(200, 400))
    r = bench.cpu_baseline(w, budget_s=0.6, sample=6, processes=2)
    assert r["cores"] == 2 and r["kind"] == "oracle"
    assert r["value"] > 0 and r["single_thread"] > 0


def _reference_arm(rank, world):
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--gpus", str(world)], cwd=root, env=env,
                       capture_output=True, text=True, timeout=300)
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    return r.returncode, [json.loads(l) for l in lines]


def test_reference_arm_rank0_prints_one_line_other_ranks_nothing():
    """The reference arm (the oracle on a bounded sample of the batch) runs on
    rank 0 alone and prints one JSON line with the contract's keys; any other
    rank exits 0 without work or output."""
    rc, out = _reference_arm(0, 2)
    assert rc == 0 and len(out) == 1
    d = out[0]
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
    assert d["metric"] == bench.METRIC and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    rc, out = _reference_arm(1, 2)
    assert rc == 0 and out == []


def test_traffic_tables_hold_positive_numbers_or_null():
    """Every measured-traffic entry is a positive number, or None once its
    kernel changed after the capture; scaling a None entry gives None."""
    import bench
    for table in (bench.MEASURED_STAGE_TRAFFIC_PER_POINT, bench.MEASURED_RUN_TRAFFIC_PER_POINT_STEP,
                  bench.MEASURED_STAGE_TRAFFIC_2D_PER_POINT,
                  bench.MEASURED_ADJOINT_TRAFFIC_PER_POINT_STEP):
        for k, v in table.items():
            assert v is None or (isinstance(v, float) and v > 0), (k, v)
            got = bench.scaled_traffic(table, k, 1000)
            assert got is None if v is None else got == v * 1000
    assert bench.scaled_traffic({"a": None}, "a", 5) is None
    assert bench.scaled_traffic({}, "a", 5) is None
