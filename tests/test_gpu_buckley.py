"""GPU parity of the Buckley-Leverett path (Example 3.4, non-convex flux,
alpha over the admissible states) against the oracle, with the tolerances of
the 1D parity tests: per stage 1e-13 of the field scales, full shocked runs
1e-8 relative L-inf; and the GPU solution's L1 error against the exact
entropy solution, which must match the oracle's."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import exact as E
from paper_2207_05258_gb300 import workloads as W
from _util import oracle_problem
from test_gpu_parity_1d import check_rhs, compare_runs, gpu_run, hw, oracle_run, split  # noqa: F401

pytestmark = pytest.mark.gpu
SIZES = [4, 5, 31, 123, 124, 125, 128, 248, 249, 400]


def bl_batch(sizes, seed, bc):
    """Ragged batch of saturations in [0, 1]: smooth waves, steps and noise."""
    rng = np.random.default_rng(seed)
    Us, Vs = [], []
    for k, n in enumerate(sizes):
        x = W.centers(-1, 1, n)
        if k % 3 == 2:
            U = np.where(np.abs(x + rng.uniform(-0.3, 0.3)) < 0.4, 0.95, 0.05)
            V = np.zeros(n)
        else:
            U = np.clip(0.5 + 0.4 * np.sin(np.pi * x + rng.uniform(0, 6)) +
                        0.03 * rng.standard_normal(n), 0.0, 1.0)
            V = 2 * rng.standard_normal(n)
        Us.append(U)
        Vs.append(V)
    return W.Workload("blb", "buckley", 1, list(sizes), 1, -1.0, 1.0, 0.0, 1.0, 0.4,
                      (bc, bc, "periodic", "periodic"), np.concatenate(Us), np.concatenate(Vs),
                      inflow=(0.9, 0, 0, 0))


@pytest.mark.parametrize("bc", ["periodic", "outflow", "inflow"])
def test_rhs_ragged(hw, bc):
    check_rhs(hw, bl_batch(SIZES, 3, bc))


@pytest.mark.parametrize("opts", [dict(limiter=0), dict(lin_w=(0.6, 0.3, 0.1))])
def test_rhs_options(hw, opts):
    check_rhs(hw, bl_batch([64, 129, 300], 4, "outflow"), **opts)


def test_one_step_ragged(hw):
    w = bl_batch(SIZES, 5, "outflow")
    compare_runs(w, gpu_run(hw, w, 1.0, steps=1), oracle_run(w, 1.0, steps=1), 1e-13, 1e-12)


@pytest.mark.parametrize("n", [80, 400])
def test_example_3_4_to_final_time(hw, n):
    w = W.buckley_leverett(n)
    g = gpu_run(hw, w, w.t_end)
    o = oracle_run(w, w.t_end)
    compare_runs(w, g, o, 1e-8, 1e-6)
    x = W.centers(-1, 1, n)
    ex = E.buckley_leverett_exact(x, w.t_end)
    eg = float(np.mean(np.abs(g[0] - ex)))
    eo = float(np.mean(np.abs(o[0][0].ravel() - ex)))
    print("Example 3.4 N=%d: L1 error GPU %.6e oracle %.6e" % (n, eg, eo))
    assert abs(eg - eo) <= 1e-8


def test_fp32_error_against_fp64_oracle(hw, record_property):
    w = W.buckley_leverett(400)
    g = gpu_run(hw, w, w.t_end, precision="fp32")
    o = oracle_run(w, w.t_end)
    e_inf = float(np.max(np.abs(g[0] - o[0][0].ravel())))
    e_1 = float(np.mean(np.abs(g[0] - o[0][0].ravel())))
    record_property("bl_fp32_linf", e_inf)
    print("Example 3.4 N=400 FP32 vs FP64 oracle: Linf %.3e L1 %.3e" % (e_inf, e_1))
    assert e_1 < 1e-4


def test_rejects_reflective_walls_and_2d(hw):
    with pytest.raises(hw.HwenoError):
        hw.Solver("buckley", 1, 40, x0=-1.0, x1=1.0, bc=("reflective",) * 4)
    with pytest.raises(hw.HwenoError):
        hw.Solver("buckley", 2, 16, 16)
