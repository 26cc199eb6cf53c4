"""Ownership of device memory at the C ABI: the library allocates all of its
scratch in hweno_create, so no later call allocates, and the calls that only
enqueue work can be recorded into a CUDA graph by the caller. Also: a graph
that hweno_run recorded is not replayed after the options or the tile
variant changed (it would hold the old scheme parameters and launch shapes).
"""
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


def _p(x):
    return None if x is None else ctypes.c_void_p(x.data_ptr())


def _subset(w, pick):
    Us, Vs = zip(*(w.instance(k) for k in pick))
    return W.Workload("sub", w.equation, 1, [w.nx[k] for k in pick], 1, w.x0, w.x1, w.y0, w.y1,
                      w.t_end, w.bc, np.concatenate([u.ravel() for u in Us]),
                      np.concatenate([v.ravel() for v in Vs]))


class _Buffers:
    """Every array the calls below need, made before the measured region so
    that torch's own allocator stays out of it."""

    def __init__(self, s, w):
        dev = "cuda"
        self.U = torch.from_numpy(w.U.copy()).to(dev)
        self.V = torch.from_numpy(w.V.copy()).to(dev)
        self.W = torch.from_numpy(w.W.copy()).to(dev) if w.dim == 2 else None
        z = lambda x: None if x is None else torch.zeros_like(x)
        self.dU, self.dV, self.dW = z(self.U), z(self.V), z(self.W)
        self.Vl, self.Wl = z(self.V), z(self.W)
        self.lU, self.lV, self.lW = z(self.U), z(self.V), z(self.W)
        self.t = torch.zeros(s.batch, dtype=torch.float64, device=dev)
        self.t0 = torch.zeros_like(self.t)
        self.dt = torch.zeros_like(self.t)
        self.tot = torch.zeros(s.batch * s.m, dtype=torch.float64, device=dev)
        self.rec = torch.zeros(s.record_bytes, dtype=torch.uint8, device=dev)
        pin = lambda x: None if x is None else x.cpu().pin_memory()
        self.hU, self.hV, self.hW = pin(self.U), pin(self.V), pin(self.W)
        self.ht = torch.zeros(s.batch, dtype=torch.float64).pin_memory()
        self.ms = (ctypes.c_double * 5)()
        self.chosen = ctypes.c_int(0)
        self.pu = ctypes.c_longlong(0)


def _exercise(hw, s, b, t_end):
    """Call every context entry point once (FP64 1D or 2D)."""
    lib, h = hw.lib, s.h
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ok = lambda rc: s._check(rc)
    ok(lib.hweno_rhs(h, _p(b.U), _p(b.V), _p(b.W), _p(b.dU), _p(b.dV), _p(b.dW), _p(b.Vl),
                     _p(b.Wl), _p(b.t), st))
    ok(lib.hweno_totals(h, _p(b.U), _p(b.tot), st))
    ok(lib.hweno_step(h, _p(b.U), _p(b.V), _p(b.W), _p(b.t), t_end, _p(b.dt), st))
    ok(lib.hweno_adjoint_step(h, _p(b.U), _p(b.V), _p(b.W), _p(b.t0), _p(b.dt), _p(b.lU),
                              _p(b.lV), _p(b.lW), st))
    ok(lib.hweno_step_record(h, _p(b.U), _p(b.V), _p(b.W), _p(b.t), t_end, _p(b.dt), _p(b.rec),
                             st))
    ok(lib.hweno_adjoint_step_recorded(h, _p(b.U), _p(b.V), _p(b.W), _p(b.rec), _p(b.t0),
                                       _p(b.dt), _p(b.lU), _p(b.lV), _p(b.lW), st))
    ok(lib.hweno_step_host(h, _p(b.hU), _p(b.hV), _p(b.hW), _p(b.ht), t_end, 2, st))
    if s.dim == 1:
        ok(lib.hweno_run_persistent(h, _p(b.U), _p(b.V), _p(b.t), t_end, 2, ctypes.byref(b.pu),
                                    st))
        ok(lib.hweno_autotune(h, _p(b.U), _p(b.V), None, _p(b.t), t_end, ctypes.byref(b.chosen),
                              b.ms, st))
        ok(lib.hweno_run_persistent(h, _p(b.U), _p(b.V), _p(b.t), t_end, 2, None, st))
    assert lib.hweno_active_instances(h, st) >= 0
    ok(lib.hweno_sync_status(h, st))


@pytest.mark.parametrize("case", ["euler1d_batch", "burgers1d", "euler2d", "euler2d_fused"])
def test_no_call_after_create_allocates_device_memory(hw, case):
    """A first context runs every call once (the first launch of a kernel
    loads its module, which takes device memory). A second context of the
    same problem is then created, and every call on it leaves the device's
    free memory unchanged: all scratch came from hweno_create."""
    if case == "euler1d_batch":
        full = W.riemann_batch(count=64, seed=5)
        w = _subset(full, list(range(64)))
    elif case == "burgers1d":
        w = W.burgers1d_sine(100000)
    else:
        w = W.euler2d_smooth(160, t_end=1.0)
    opts = {"fused_2d": 1} if case == "euler2d_fused" else {}
    t_end = float(w.t_end)
    warm = hw.Solver.from_workload(w, **opts)
    bw = _Buffers(warm, w)
    _exercise(hw, warm, bw, t_end)
    s = hw.Solver.from_workload(w, **opts)
    b = _Buffers(s, w)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    _exercise(hw, s, b, t_end)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0 - free1)
    # the adjoint scratch made by create is large enough to show in the count
    adj = 8 * s.m * s.num_points * (6 if w.dim == 1 else 12)
    assert adj >= 4 << 20


@pytest.mark.parametrize("fused_small", [0, 2])
def test_persistent_run_recorded_into_a_graph_replays_the_same_bits(hw, fused_small):
    """hweno_run_persistent without a point-update count only enqueues work
    (counter resets, one wave-speed launch, one persistent launch): recorded
    into a CUDA graph on a fresh context and replayed twice, it gives the
    bits of two direct calls."""
    full = W.riemann_batch(count=24, seed=8)
    if fused_small == 2:
        w = _subset(full, [k for k in range(24) if full.nx[k] <= 800][:4])
    else:
        w = _subset(full, list(range(24)))
    K = 3
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        s = hw.Solver.from_workload(w, fused_small=fused_small)
        U = torch.from_numpy(w.U.copy()).cuda()
        V = torch.from_numpy(w.V.copy()).cuda()
        t = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
    side.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="thread_local"):
        s.run_persistent(U, V, t, w.t_end, K, count=False)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    s.sync_status()
    r = hw.Solver.from_workload(w, fused_small=fused_small)
    U2 = torch.from_numpy(w.U.copy()).cuda()
    V2 = torch.from_numpy(w.V.copy()).cuda()
    t2 = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
    r.run_persistent(U2, V2, t2, w.t_end, K)
    r.run_persistent(U2, V2, t2, w.t_end, K)
    torch.cuda.synchronize()
    assert torch.all(t > 0)
    assert torch.equal(U, U2) and torch.equal(V, V2) and torch.equal(t, t2)


def test_step_recorded_into_a_graph_replays_the_same_bits(hw):
    """hweno_step (five launches and two memsets in 1D) recorded by the caller
    into a CUDA graph gives the bits of direct calls."""
    full = W.riemann_batch(count=16, seed=12)
    w = _subset(full, list(range(16)))
    s = hw.Solver.from_workload(w)
    U = torch.from_numpy(w.U.copy()).cuda()
    V = torch.from_numpy(w.V.copy()).cuda()
    t = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="thread_local"):
        s.step(U, V, None, t, w.t_end)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    r = hw.Solver.from_workload(w)
    U2 = torch.from_numpy(w.U.copy()).cuda()
    V2 = torch.from_numpy(w.V.copy()).cuda()
    t2 = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
    for _ in range(3):
        r.step(U2, V2, None, t2, w.t_end)
    torch.cuda.synchronize()
    assert torch.equal(U, U2) and torch.equal(V, V2) and torch.equal(t, t2)


@pytest.mark.parametrize("change", ["cfl", "tile_variant", "autotune"])
def test_hweno_run_records_again_after_options_change(hw, change):
    """hweno_run keeps its recorded graph for the same arrays; after
    hweno_set_options or hweno_autotune the next hweno_run must record the
    new scheme (here compared with plain hweno_step calls that make the same
    change at the same point)."""
    full = W.riemann_batch(count=16, seed=21)
    w = _subset(full, list(range(16)))
    side = torch.cuda.Stream()

    def apply(s, U, V, t):
        if change == "cfl":
            s.set_options(cfl=0.3)
        elif change == "tile_variant":
            s.set_options(tile_variant=3)
        else:
            s.autotune(U, V, None, t, w.t_end)

    with torch.cuda.stream(side):
        s = hw.Solver.from_workload(w)
        U = torch.from_numpy(w.U.copy()).cuda()
        V = torch.from_numpy(w.V.copy()).cuda()
        t = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
        s.run_graph(U, V, None, t, w.t_end, max_steps=2, steps_per_launch=2)
        apply(s, U, V, t)
        s.run_graph(U, V, None, t, w.t_end, max_steps=2, steps_per_launch=2)
        r = hw.Solver.from_workload(w)
        U2 = torch.from_numpy(w.U.copy()).cuda()
        V2 = torch.from_numpy(w.V.copy()).cuda()
        t2 = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
        for _ in range(2):
            r.step(U2, V2, None, t2, w.t_end)
        apply(r, U2, V2, t2)
        for _ in range(2):
            r.step(U2, V2, None, t2, w.t_end)
    side.synchronize()
    assert torch.equal(U, U2) and torch.equal(V, V2) and torch.equal(t, t2)


@pytest.mark.parametrize("fused_2d", [0, 1])
def test_2d_step_recorded_into_a_graph_replays_the_same_bits(hw, fused_2d):
    """hweno_step in 2D (eight launches split, five fused) recorded by the
    caller into a CUDA graph gives the bits of direct calls."""
    w = W.euler2d_smooth(96, ny=40, t_end=1.0)
    dev = lambda x: torch.from_numpy(x.copy()).cuda()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        s = hw.Solver.from_workload(w, fused_2d=fused_2d)
        U, V, Wd = dev(w.U), dev(w.V), dev(w.W)
        t = torch.zeros(1, dtype=torch.float64, device="cuda")
    side.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="thread_local"):
        s.step(U, V, Wd, t, w.t_end)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    s.sync_status()
    r = hw.Solver.from_workload(w, fused_2d=fused_2d)
    U2, V2, W2 = dev(w.U), dev(w.V), dev(w.W)
    t2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(3):
        r.step(U2, V2, W2, t2, w.t_end)
    torch.cuda.synchronize()
    assert r.launches_last_call == (5 if fused_2d else 8)
    assert torch.equal(U, U2) and torch.equal(V, V2) and torch.equal(Wd, W2)
    assert torch.equal(t, t2)


def test_2d_hweno_run_records_again_after_the_stage_form_changes(hw):
    """hweno_run in 2D: after hweno_set_options switches the stage form the
    next hweno_run records the fused launches (compared with plain steps
    that switch at the same point)."""
    w = W.euler2d_smooth(64, ny=48, t_end=1.0)
    dev = lambda x: torch.from_numpy(x.copy()).cuda()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        s = hw.Solver.from_workload(w, dt_mode=1)
        U, V, Wd = dev(w.U), dev(w.V), dev(w.W)
        t = torch.zeros(1, dtype=torch.float64, device="cuda")
        s.run_graph(U, V, Wd, t, w.t_end, max_steps=2, steps_per_launch=2)
        s.set_options(dt_mode=1, fused_2d=1)
        s.run_graph(U, V, Wd, t, w.t_end, max_steps=2, steps_per_launch=2)
        r = hw.Solver.from_workload(w, dt_mode=1)
        U2, V2, W2 = dev(w.U), dev(w.V), dev(w.W)
        t2 = torch.zeros(1, dtype=torch.float64, device="cuda")
        for _ in range(2):
            r.step(U2, V2, W2, t2, w.t_end)
        r.set_options(dt_mode=1, fused_2d=1)
        for _ in range(2):
            r.step(U2, V2, W2, t2, w.t_end)
        assert r.launches_last_call == 5
    side.synchronize()
    assert torch.equal(U, U2) and torch.equal(V, V2) and torch.equal(Wd, W2)
    assert torch.equal(t, t2)
