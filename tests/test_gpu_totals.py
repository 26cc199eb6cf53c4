"""hweno_totals: FP64 conserved totals sum_i U_c dx (dy) with a fixed
summation order. Checked against numpy sums, for run-to-run bit equality, and
for discrete conservation over periodic runs (the flux form of Eq. odeH and
Eq. ode2H conserves them to rounding)."""
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


def ref_totals(w, U):
    out = []
    if w.dim == 2:
        U = U.reshape(w.m, -1)
        return U.sum(axis=1)[None, :] * ((w.x1 - w.x0) / w.nx[0]) * ((w.y1 - w.y0) / w.ny)
    off = 0
    for n in w.nx:
        out.append(U[off:off + w.m * n].reshape(w.m, n).sum(axis=1) * ((w.x1 - w.x0) / n))
        off += w.m * n
    return np.array(out)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_totals_of_a_ragged_batch(hw, precision):
    w = W.riemann_batch(count=37, seed=4)
    s = hw.Solver.from_workload(w, precision=precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    U = torch.from_numpy(w.U).to("cuda", dt)
    a = s.totals(U).cpu().numpy()
    b = s.totals(U).cpu().numpy()
    assert np.array_equal(a, b)
    ref = ref_totals(w, U.double().cpu().numpy())
    assert np.max(np.abs(a - ref) / np.abs(ref)) < 1e-13


@pytest.mark.parametrize("make", [lambda: W.burgers1d_sine(400),
                                  lambda: W.euler2d_smooth(64, dt_mode="cfl"),
                                  lambda: W.burgers2d_sine(48, dt_mode="cfl")],
                         ids=["burgers1d", "euler2d", "burgers2d"])
def test_periodic_runs_conserve_totals(hw, make):
    w = make()
    s = hw.Solver.from_workload(w)
    U = torch.from_numpy(w.U.copy()).cuda()
    V = torch.from_numpy(w.V.copy()).cuda()
    Wd = torch.from_numpy(w.W.copy()).cuda() if w.dim == 2 else None
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    t0 = s.totals(U).cpu().numpy()
    for _ in range(20):
        s.step(U, V, Wd, t, 10.0)
    s.sync_status()
    t1 = s.totals(U).cpu().numpy()
    scale = ref_totals(w, np.abs(w.U))
    assert np.all(np.abs(t1 - t0) <= 1e-13 * scale), (t1 - t0) / scale
