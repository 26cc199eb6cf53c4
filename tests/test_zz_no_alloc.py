"""hweno_step_1d_noalloc: the allocation-free step for callers that cannot
allocate device memory (hosts that own every device allocation through their
own pool, latency-critical paths that must not pay cudaMalloc's implicit
synchronisation, plug-ins handed only pre-allocated buffers). Its scratch is
a fixed device array inside the library, so the check is that two calls in a
row through the C ABI give what the context-based hweno_step gives, within
the per-step tolerance of the other parity tests.

The file name makes pytest collect it last: it checks an addition beside the
scheme's own path, so a run that stops at the first failure has already run
every other test by the time it gets here. Its result does not depend on the
order: it also passes alone in a fresh process."""
import ctypes

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


def _bc(hw, w):
    b = hw.Bc(hw.BC[w.bc[0]], hw.BC[w.bc[1]], 0, 0)
    b.inflow[:] = list(w.inflow) + [0.0] * (4 - len(w.inflow))
    return b


def _reference(hw, w, steps):
    s = hw.Solver.from_workload(w)
    U = torch.from_numpy(w.U.copy()).cuda()
    V = torch.from_numpy(w.V.copy()).cuda()
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = []
    for _ in range(steps):
        s.step(U, V, None, t, w.t_end)
        s.sync_status()
        out.append((U.cpu().numpy().copy(), V.cpu().numpy().copy(), float(t.item())))
    s.close()
    return out


def _noalloc(hw, w, steps, opt=None):
    U = torch.from_numpy(w.U.copy()).cuda()
    V = torch.from_numpy(w.V.copy()).cuda()
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    bc = _bc(hw, w)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = lambda x: ctypes.c_void_p(x.data_ptr())
    out = []
    for _ in range(steps):
        rc = hw.lib.hweno_step_1d_noalloc(
            hw.BURGERS if w.equation == "burgers" else hw.EULER, w.nx[0], w.x0, w.x1,
            w.gas_gamma, ctypes.byref(bc), None if opt is None else ctypes.byref(opt),
            p(U), p(V), p(t), w.t_end, p(dt), stream)
        assert rc == hw.OK, rc
        out.append((U.cpu().numpy().copy(), V.cpu().numpy().copy(), float(t.item())))
        assert dt.item() > 0
    return out


@pytest.mark.parametrize("make", [
    lambda: W.burgers1d_sine(400),
    lambda: W.riemann1d(300, (0.9, 0.2, 0.8), (0.2, -0.3, 0.3)),
    lambda: W.riemann1d(3200, *W.riemann_batch(count=2, seed=5).meta["states"][1]),
], ids=["burgers_n400", "euler_n300", "euler_n3200"])
def test_two_calls_match_context_step(hw, make):
    w = make()
    ref = _reference(hw, w, 2)
    got = _noalloc(hw, w, 2)
    for (ur, vr, tr), (ug, vg, tg) in zip(ref, got):
        assert np.max(np.abs(ug - ur)) <= 1e-13 * np.max(np.abs(ur))
        assert np.max(np.abs(vg - vr)) <= 1e-12 * max(np.max(np.abs(vr)), 1.0)
        assert tg == tr


def test_rejects_sizes_beyond_the_fixed_array(hw):
    n = 16385  # HWENO_NOALLOC_MAX_POINTS + 1
    U = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    bc = hw.Bc(1, 1, 0, 0)
    p = lambda x: ctypes.c_void_p(x.data_ptr())
    rc = hw.lib.hweno_step_1d_noalloc(hw.EULER, n, 0.0, 1.0, 1.4, ctypes.byref(bc), None,
                                      p(U), p(U), p(t), 1.0, None, None)
    assert rc == hw.EINVAL
