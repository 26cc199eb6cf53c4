"""The FP32 path's error, stated per result at the benchmark workloads' sizes.

The FP32 kernels keep the state and the reconstruction in FP32 (wave
speeds, time steps and times in FP64). Each test runs a workload to its
final time in FP32 and in FP64 on the GPU (the FP64 path is pinned to the
oracle at these sizes by test_gpu_full_size.py) and states the difference;
the smooth problem is also compared with its exact solution. The bounds are
about ten times the measured values.
"""
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


def run_to_end(hw, w, precision, t_end):
    s = hw.Solver.from_workload(w, precision=precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    U = torch.from_numpy(w.U.copy()).to("cuda", dt)
    V = torch.from_numpy(w.V.copy()).to("cuda", dt)
    Wd = torch.from_numpy(w.W.copy()).to("cuda", dt) if w.dim == 2 else None
    t = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
    s.run(U, V, Wd, t, t_end)
    s.sync_status()
    assert torch.all(t == t_end)
    out = U.double().cpu().numpy()
    s.close()
    return out


def test_fp32_riemann_batch_to_final_time(hw, record_property):
    """2048 Riemann problems (N = 200..3200) to T = 0.15: per-instance L1
    difference of the density, FP32 against FP64, relative to the FP64
    density's L1 norm."""
    w = W.riemann_batch(count=2048)
    g64 = run_to_end(hw, w, "fp64", w.t_end)
    g32 = run_to_end(hw, w, "fp32", w.t_end)
    rel = []
    for k, n in enumerate(w.nx):
        o = 3 * int(w.offsets[k])
        r64, r32 = g64[o:o + n], g32[o:o + n]
        rel.append(np.abs(r32 - r64).sum() / np.abs(r64).sum())
    rel = np.array(rel)
    record_property("fp32_riemann_rel_l1_max", float(rel.max()))
    record_property("fp32_riemann_rel_l1_median", float(np.median(rel)))
    print("FP32 Riemann batch T=0.15: rel L1(rho) vs FP64 max %.2e median %.2e"
          % (rel.max(), np.median(rel)))
    assert rel.max() < 4e-4 and np.median(rel) < 3e-5  # measured 3.8e-5, 2.3e-6


def test_fp32_smooth_2d_against_the_exact_solution(hw, record_property):
    """2D Euler density wave, 256^2, to T = 2 (one period: the exact solution
    is the initial data): FP32 and FP64 errors of the density."""
    w = W.euler2d_smooth(256, dt_mode="cfl")
    exact = w.U.reshape(4, 256, 256)[0]
    errs = {}
    for prec in ("fp64", "fp32"):
        g = run_to_end(hw, w, prec, w.t_end).reshape(4, 256, 256)[0]
        errs[prec] = (np.abs(g - exact).max() / np.abs(exact).max(),
                      np.abs(g - exact).mean() / np.abs(exact).mean())
        record_property(prec + "_smooth2d_256_rel_linf", float(errs[prec][0]))
    print("2D smooth 256^2 T=2 vs exact: FP64 rel Linf %.2e L1 %.2e; FP32 rel Linf %.2e L1 %.2e"
          % (errs["fp64"] + errs["fp32"]))
    assert errs["fp64"][0] < 3e-8  # measured 3.0e-9
    assert errs["fp32"][0] < 4e-4  # measured 3.6e-5


def test_fp32_double_mach(hw, record_property):
    """Double Mach reflection, 1920 x 480, to T = 0.02: L1 difference of the
    density, FP32 against FP64, relative to the FP64 density's L1 norm."""
    w = W.double_mach(1920, 480, t_end=0.02)
    r64 = run_to_end(hw, w, "fp64", w.t_end).reshape(4, 480, 1920)[0]
    r32 = run_to_end(hw, w, "fp32", w.t_end).reshape(4, 480, 1920)[0]
    rel = np.abs(r32 - r64).sum() / np.abs(r64).sum()
    record_property("fp32_double_mach_rel_l1", float(rel))
    print("FP32 double Mach 1920x480 T=0.02: rel L1(rho) vs FP64 %.2e" % rel)
    assert rel < 2e-5  # measured 1.9e-6
