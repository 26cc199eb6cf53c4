"""Python binding of the C ABI in include/hweno.h (ctypes; argument
marshalling only: every step of the scheme runs in the CUDA library).

Arrays are torch CUDA tensors (float64 for HWENO_FP64, float32 for
HWENO_FP32), contiguous, laid out [instance][component][j][i]. Work is
enqueued on torch's current stream. Importing this module loads
``_build/libhweno.so`` and raises if it is missing: there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
# HWENO_LIBRARY selects another build of the library (the checked build of
# the tests: _build_checked/libhweno.so)
LIB_PATH = os.environ.get("HWENO_LIBRARY") or os.path.join(_PKG, "_build", "libhweno.so")

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, ENOTSUP, EBOUNDS = 0, -1, -2, -3, -4, -5, -6, -7
BURGERS, EULER, BUCKLEY = 0, 1, 2
EQUATIONS = dict(burgers=BURGERS, euler=EULER, buckley=BUCKLEY)
FP64, FP32 = 0, 1
TILE_VARIANTS = 5  # HWENO_TILE_VARIANTS: 1D tile shapes
MAX_SIZE_CLASSES = 16  # HWENO_MAX_SIZE_CLASSES
CLUSTER_MAX_POINTS = 992  # HWENO_CLUSTER_MAX_POINTS: fused_small = 2
BC = dict(periodic=0, outflow=1, reflective=2, inflow=3, dmr_bottom=4, dmr_top=5)
_NAMES = {EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA", ENONFINITE: "ENONFINITE",
          ETIMEOUT: "ETIMEOUT", ENOTSUP: "ENOTSUP", EBOUNDS: "EBOUNDS"}


class HwenoError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_NAMES.get(code, "error"), code, msg))
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y0", ctypes.c_double), ("y1", ctypes.c_double),
                ("batch", ctypes.c_int), ("nx_per_instance", ctypes.POINTER(ctypes.c_int)),
                ("precision", ctypes.c_int)]


class Bc(ctypes.Structure):
    _fields_ = [("xlo", ctypes.c_int), ("xhi", ctypes.c_int), ("ylo", ctypes.c_int),
                ("yhi", ctypes.c_int), ("inflow", ctypes.c_double * 4),
                ("pre", ctypes.c_double * 4), ("dmr_x0", ctypes.c_double),
                ("dmr_speed", ctypes.c_double), ("dmr_angle", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("lin_w", ctypes.c_double * 3), ("lim_d", ctypes.c_double * 3),
                ("eps", ctypes.c_double), ("cfl", ctypes.c_double), ("dt_mode", ctypes.c_int),
                ("dt_fixed", ctypes.c_double), ("limiter", ctypes.c_int),
                ("eig_avg", ctypes.c_int), ("tile_variant", ctypes.c_int),
                ("fused_small", ctypes.c_int), ("adj_frozen_weights", ctypes.c_int),
                ("fused_2d", ctypes.c_int)]


_VP = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes); every entry point declared in include/hweno.h
SIGNATURES = {
    "hweno_default_options": (ctypes.c_int, [ctypes.POINTER(Options)]),
    "hweno_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, ctypes.POINTER(Grid),
                                    ctypes.c_double, ctypes.POINTER(Bc)]),
    "hweno_set_options": (ctypes.c_int, [_VP, ctypes.POINTER(Options)]),
    "hweno_rhs": (ctypes.c_int, [_VP] + [_VP] * 8 + [_VP, _VP]),
    "hweno_step": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.c_double, _VP, _VP]),
    "hweno_step_host": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.c_double, ctypes.c_int,
                                       _VP]),
    "hweno_run": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.c_double, ctypes.c_longlong,
                                 ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                 ctypes.POINTER(ctypes.c_longlong), _VP]),
    "hweno_totals": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "hweno_size_classes": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int)]),
    "hweno_autotune_classes": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_double,
                                              ctypes.POINTER(ctypes.c_int), _DP, _VP]),
    "hweno_set_class_variants": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int)]),
    "hweno_autotune": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.c_double,
                                      ctypes.POINTER(ctypes.c_int), _DP, _VP]),
    "hweno_adjoint_step": (ctypes.c_int, [_VP] * 10),
    "hweno_test_inject": (ctypes.c_int, [_VP, ctypes.c_int]),
    "hweno_run_persistent": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_double, ctypes.c_int,
                                            _VP, _VP]),
    "hweno_sync_status": (ctypes.c_int, [_VP, _VP]),
    "hweno_num_points": (ctypes.c_longlong, [_VP]),
    "hweno_active_instances": (ctypes.c_int, [_VP, _VP]),
    "hweno_launches_last_call": (ctypes.c_int, [_VP]),
    "hweno_get_options": (ctypes.c_int, [_VP, ctypes.POINTER(Options)]),
    "hweno_profile_start": (ctypes.c_int, [_VP, ctypes.c_int]),
    "hweno_profile_read": (ctypes.c_int, [_VP, _DP, ctypes.POINTER(ctypes.c_int), _VP]),
    "hweno_step_1d_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, ctypes.POINTER(Bc),
                                             ctypes.POINTER(Options), _VP, _VP, _VP,
                                             ctypes.c_double, _VP, _VP]),
    "hweno_measure_fp64_peak": (ctypes.c_int, [_DP, _VP]),
    "hweno_adjoint_record_bytes": (ctypes.c_longlong, [_VP]),
    "hweno_step_record": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.c_double, _VP, _VP,
                                         _VP]),
    "hweno_adjoint_step_recorded": (ctypes.c_int, [_VP] * 11),
    "hweno_last_error": (ctypes.c_char_p, [_VP]),
    "hweno_destroy": (ctypes.c_int, [_VP]),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libhweno.so not built (%s); run python -m paper_2207_05258_gb300.build"
                          % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype, fn.argtypes = res, args
    return lib


lib = _load()


def default_options() -> Options:
    o = Options()
    lib.hweno_default_options(ctypes.byref(o))
    return o


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def measure_fp64_peak() -> float:
    """hweno_measure_fp64_peak: FP64 TFLOP/s of a DFMA-only loop on the
    current device (the ceiling that FP64-pipe-bound kernels can reach)."""
    out = ctypes.c_double(0.0)
    rc = lib.hweno_measure_fp64_peak(ctypes.byref(out), _stream())
    if rc != OK:
        raise HwenoError(rc, "hweno_measure_fp64_peak failed")
    return out.value


class Solver:
    """One L-HWENO problem (or a ragged 1D batch) bound to a library context."""

    def __init__(self, equation: str, dim: int, nx: Sequence[int] | int, ny: int = 1,
                 x0: float = 0.0, x1: float = 1.0, y0: float = 0.0, y1: float = 1.0,
                 gamma: float = 1.4, bc=("periodic",) * 4, inflow=(0, 0, 0, 0),
                 pre=(0, 0, 0, 0), dmr_x0=1.0 / 6.0, dmr_speed=10.0, dmr_angle=1.0471975511965976,
                 precision: str = "fp64", **options):
        nxs = [int(nx)] if isinstance(nx, int) else [int(n) for n in nx]
        self.equation, self.dim, self.nx, self.ny = equation, dim, nxs, (ny if dim == 2 else 1)
        self.batch = len(nxs) if dim == 1 else 1
        self.m = (3 if dim == 1 else 4) if equation == "euler" else 1
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self._nx_arr = (ctypes.c_int * len(nxs))(*nxs)
        g = Grid(dim, nxs[0], self.ny, x0, x1, y0, y1, self.batch,
                 ctypes.cast(self._nx_arr, ctypes.POINTER(ctypes.c_int)),
                 FP64 if precision == "fp64" else FP32)
        b = Bc(*(BC[s] for s in bc))
        b.inflow[:] = list(inflow) + [0.0] * (4 - len(inflow))
        b.pre[:] = list(pre) + [0.0] * (4 - len(pre))
        b.dmr_x0, b.dmr_speed, b.dmr_angle = dmr_x0, dmr_speed, dmr_angle
        h = ctypes.c_void_p()
        rc = lib.hweno_create(ctypes.byref(h), EQUATIONS[equation],
                              ctypes.byref(g), gamma, ctypes.byref(b))
        if rc != OK:
            raise HwenoError(rc, "hweno_create failed")
        self.h = h
        if options:
            self.set_options(**options)

    @classmethod
    def from_workload(cls, w, precision="fp64", **options):
        dt_mode = options.pop("dt_mode", 1 if w.dt_mode == "accuracy" else 0)
        return cls(w.equation, w.dim, w.nx if w.dim == 1 else w.nx[0], w.ny, w.x0, w.x1, w.y0,
                   w.y1, w.gas_gamma, w.bc, w.inflow, w.pre, w.dmr_x0, w.dmr_speed, w.dmr_angle,
                   precision=precision, dt_mode=dt_mode, **options)

    def _check(self, rc):
        if rc != OK:
            raise HwenoError(rc, lib.hweno_last_error(self.h).decode())

    def options(self) -> "Options":
        """hweno_get_options: the context's current options."""
        o = Options()
        self._check(lib.hweno_get_options(self.h, ctypes.byref(o)))
        return o

    def set_options(self, **kw):
        """Change the named options; the others keep their current values
        (including a tile variant or 2D stage form chosen by the autotuner)."""
        o = self.options()
        for k, v in kw.items():
            if k in ("lin_w", "lim_d"):
                getattr(o, k)[:] = list(v)
            else:
                if not hasattr(o, k):
                    raise AttributeError("unknown option %r" % k)
                setattr(o, k, v)
        self._check(lib.hweno_set_options(self.h, ctypes.byref(o)))

    @property
    def num_points(self) -> int:
        return int(lib.hweno_num_points(self.h))

    def state_shape(self):
        return (self.m * self.num_points,)

    def rhs(self, U, V, W=None, t=None, limited=True):
        """L^1, L^2 (, L^3) and the limited derivatives at state (U, V, W)."""
        t = torch.zeros(self.batch, dtype=torch.float64, device=U.device) if t is None else t
        dU, dV = torch.empty_like(U), torch.empty_like(V)
        dW = torch.empty_like(W) if W is not None else None
        Vl = torch.empty_like(V) if limited else None
        Wl = torch.empty_like(W) if (limited and W is not None) else None
        self._check(lib.hweno_rhs(self.h, _ptr(U), _ptr(V), _ptr(W), _ptr(dU), _ptr(dV), _ptr(dW),
                                  _ptr(Vl), _ptr(Wl), _ptr(t), _stream()))
        out = dict(L1=dU, L2=dV, Vt=Vl)
        if W is not None:
            out.update(L3=dW, Wt=Wl)
        return out

    def step(self, U, V, W=None, t=None, t_end=float("inf"), dt_used=None):
        """One SSP-RK3 step in place; t (float64 CUDA tensor [batch]) advances."""
        self._check(lib.hweno_step(self.h, _ptr(U), _ptr(V), _ptr(W), _ptr(t), float(t_end),
                                   _ptr(dt_used), _stream()))

    def step_host(self, U, V, W, t, t_end, nsteps=1):
        """hweno_step_host on host (ideally pinned) CPU tensors."""
        for x in (U, V, t) + ((W,) if W is not None else ()):
            if x.is_cuda or not x.is_contiguous():
                raise ValueError("expected contiguous host tensors")
        p = lambda x: None if x is None else ctypes.c_void_p(x.data_ptr())
        self._check(lib.hweno_step_host(self.h, p(U), p(V), p(W), p(t), float(t_end), nsteps,
                                        _stream()))

    def autotune(self, U, V, W=None, t=None, t_end=float("inf")):
        """hweno_autotune: returns (chosen variant, per-variant ms)."""
        t = torch.zeros(self.batch, dtype=torch.float64, device=U.device) if t is None else t
        chosen = ctypes.c_int(0)
        ms = (ctypes.c_double * TILE_VARIANTS)()
        self._check(lib.hweno_autotune(self.h, _ptr(U), _ptr(V), _ptr(W), _ptr(t), float(t_end),
                                       ctypes.byref(chosen), ms, _stream()))
        return chosen.value, list(ms)

    def size_classes(self):
        """hweno_size_classes: [(smallest, largest instance size)] per class."""
        lo = (ctypes.c_int * MAX_SIZE_CLASSES)()
        hi = (ctypes.c_int * MAX_SIZE_CLASSES)()
        n = lib.hweno_size_classes(self.h, lo, hi)
        if n < 0:
            self._check(n)
        return [(lo[i], hi[i]) for i in range(n)]

    def autotune_classes(self, U, V, t=None, t_end=float("inf")):
        """hweno_autotune_classes: returns (variant per class, per class the
        best ms of each variant)."""
        t = torch.zeros(self.batch, dtype=torch.float64, device=U.device) if t is None else t
        nq = len(self.size_classes())
        chosen = (ctypes.c_int * MAX_SIZE_CLASSES)()
        ms = (ctypes.c_double * (MAX_SIZE_CLASSES * TILE_VARIANTS))()
        self._check(lib.hweno_autotune_classes(self.h, _ptr(U), _ptr(V), _ptr(t), float(t_end),
                                               chosen, ms, _stream()))
        return ([chosen[q] for q in range(nq)],
                [[ms[q * TILE_VARIANTS + v] for v in range(TILE_VARIANTS)] for q in range(nq)])

    def set_class_variants(self, variants):
        """hweno_set_class_variants: the tile variant of each size class."""
        arr = (ctypes.c_int * MAX_SIZE_CLASSES)(*variants)
        self._check(lib.hweno_set_class_variants(self.h, arr))

    def totals(self, U):
        """FP64 conserved totals, tensor [batch, m] (fixed summation order)."""
        out = torch.empty(self.batch, self.m, dtype=torch.float64, device=U.device)
        self._check(lib.hweno_totals(self.h, _ptr(U), _ptr(out), _stream()))
        return out

    def adjoint_step(self, U, V, W, dt, lamU, lamV, lamW=None, t=None, record=None):
        """hweno_adjoint_step: lamU, lamV (, lamW) (in: d J / d output of the
        step taken from U, V (, W) at time t with time steps dt) become
        d J / d input, in place. With `record` (from step_record of that
        step): hweno_adjoint_step_recorded, no replay of the stages."""
        if record is None:
            self._check(lib.hweno_adjoint_step(self.h, _ptr(U), _ptr(V), _ptr(W), _ptr(t),
                                               _ptr(dt), _ptr(lamU), _ptr(lamV), _ptr(lamW),
                                               _stream()))
        else:
            self._check(lib.hweno_adjoint_step_recorded(
                self.h, _ptr(U), _ptr(V), _ptr(W), _ptr(record), _ptr(t), _ptr(dt), _ptr(lamU),
                _ptr(lamV), _ptr(lamW), _stream()))

    @property
    def record_bytes(self) -> int:
        """hweno_adjoint_record_bytes: size of one step record."""
        return int(lib.hweno_adjoint_record_bytes(self.h))

    def new_record(self, device="cuda"):
        """A device buffer for one step record."""
        return torch.empty(self.record_bytes, dtype=torch.uint8, device=device)

    def step_record(self, U, V, W, t, t_end, record, dt_used=None):
        """hweno_step_record: hweno_step that also saves the stage states and
        wave speeds of the step into `record` (see new_record)."""
        self._check(lib.hweno_step_record(self.h, _ptr(U), _ptr(V), _ptr(W), _ptr(t),
                                          float(t_end), _ptr(dt_used), _ptr(record), _stream()))

    def active_instances(self) -> int:
        n = lib.hweno_active_instances(self.h, _stream())
        if n < 0:
            self._check(n)
        return n

    def sync_status(self):
        self._check(lib.hweno_sync_status(self.h, _stream()))

    @property
    def launches_last_call(self) -> int:
        return int(lib.hweno_launches_last_call(self.h))

    def profile_start(self, capacity: int):
        """Bracket the next `capacity` kernel launches with CUDA events."""
        self._check(lib.hweno_profile_start(self.h, int(capacity)))

    def profile_read(self):
        """{kind: (total_ms, launches)} for kinds alpha, stage, finalize."""
        ms = (ctypes.c_double * 3)()
        n = (ctypes.c_int * 3)()
        self._check(lib.hweno_profile_read(self.h, ms, n, _stream()))
        return {k: (ms[i], n[i]) for i, k in enumerate(("alpha", "stage", "finalize"))}

    def close(self):
        if getattr(self, "h", None):
            lib.hweno_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run_graph(self, U, V, W=None, t=None, t_end=1.0, max_steps=1 << 40, steps_per_launch=32):
        """hweno_run on torch's current stream (which must not be the legacy
        default stream): returns (steps launched, point-updates)."""
        steps, pu = ctypes.c_longlong(0), ctypes.c_longlong(0)
        self._check(lib.hweno_run(self.h, _ptr(U), _ptr(V), _ptr(W), _ptr(t), float(t_end),
                                  int(max_steps), int(steps_per_launch), ctypes.byref(steps),
                                  ctypes.byref(pu), _stream()))
        return steps.value, pu.value

    def test_inject(self, kind: int):
        """hweno_test_inject (failure-detection tests)."""
        self._check(lib.hweno_test_inject(self.h, int(kind)))

    def run_persistent(self, U, V, t, t_end, steps, count=True):
        """hweno_run_persistent: `steps` steps of a 1D batch in one persistent
        launch; returns the point-updates (synchronising) when count is True."""
        pu = ctypes.c_longlong(0)
        self._check(lib.hweno_run_persistent(self.h, _ptr(U), _ptr(V), _ptr(t), float(t_end),
                                             int(steps), ctypes.byref(pu) if count else None,
                                             _stream()))
        return pu.value if count else None

    def run(self, U, V, W=None, t=None, t_end=1.0, max_steps=1 << 30, check_every=64):
        """Steps until every instance reaches t_end; returns the steps taken."""
        k = 0
        while k < max_steps:
            n = min(check_every, max_steps - k)
            for _ in range(n):
                self.step(U, V, W, t, t_end)
            k += n
            if self.active_instances() == 0:
                break
        self.sync_status()
        return k
