"""Oracle for the fifth-order finite-difference L-HWENO scheme (Zhang & Zhao,
arXiv:2207.05258): a plain FP64 CPU statement of the scheme of Sec. 2.

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline legs of ``bench.py`` may import this package. It shares no code with
the CUDA library and never imports it. The arithmetic lives in
``hweno_oracle.cpp`` (built here with g++, no FMA contraction, no fast-math);
this module only marshals numpy arrays through ctypes.

Array layout: one FP64 numpy array per field, shape (m, nx) in 1D and
(m, ny, nx) in 2D, m = 1 (Burgers), 3 (Euler 1D) or 4 (Euler 2D).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hweno_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

EQ_BURGERS, EQ_EULER, EQ_BUCKLEY = 0, 1, 2
BC_PERIODIC, BC_OUTFLOW, BC_REFLECTIVE, BC_INFLOW, BC_DMR_BOTTOM, BC_DMR_TOP = range(6)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (if stale)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Problem(ctypes.Structure):
    _fields_ = [
        ("eq", ctypes.c_int), ("dim", ctypes.c_int),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("gas_gamma", ctypes.c_double),
        ("bc", ctypes.c_int * 4),
        ("inflow", ctypes.c_double * 4), ("pre", ctypes.c_double * 4),
        ("dmr_x0", ctypes.c_double), ("dmr_speed", ctypes.c_double),
        ("dmr_angle", ctypes.c_double),
        ("lin_w", ctypes.c_double * 3), ("lim_d", ctypes.c_double * 3),
        ("eps", ctypes.c_double), ("cfl", ctypes.c_double),
        ("dt_mode", ctypes.c_int), ("dt_fixed", ctypes.c_double),
        ("limiter", ctypes.c_int), ("eig_avg", ctypes.c_int),
        ("alpha_fixed", ctypes.c_double), ("freeze_weights", ctypes.c_int),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_P = ctypes.POINTER(Problem)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.or_ncomp.argtypes = [_P]
            L.or_ncomp.restype = ctypes.c_int
            L.or_hweno_face.argtypes = [ctypes.c_int, _D, _D, ctypes.c_double, _D,
                                        ctypes.c_double, _D]
            L.or_limiter.argtypes = [ctypes.c_double] * 6 + [_D, ctypes.c_double, _D]
            L.or_hweno_face_tangent.argtypes = [ctypes.c_int, _D, _D, _D, _D, ctypes.c_double,
                                                _D, ctypes.c_double, ctypes.c_int, _D]
            L.or_limiter_tangent.argtypes = [ctypes.c_double] * 5 + [_D, ctypes.c_double, _D,
                                                                      ctypes.c_double, ctypes.c_int]
            L.or_limiter_tangent.restype = ctypes.c_double
            L.or_flux.argtypes = [_P, ctypes.c_int, _D, _D]
            L.or_jvp.argtypes = [_P, ctypes.c_int, _D, _D, _D]
            L.or_bl_alpha01.argtypes = []
            L.or_bl_alpha01.restype = ctypes.c_double
            L.or_wave_speed.argtypes = [_P, ctypes.c_int, _D]
            L.or_wave_speed.restype = ctypes.c_double
            L.or_eigen.argtypes = [_P, ctypes.c_int, _D, _D, _D, _D, _D]
            L.or_rhs_1d.argtypes = [_P, _D, _D, ctypes.c_double, _D, _D, _D, _D]
            L.or_rhs_2d.argtypes = [_P, _D, _D, _D, ctypes.c_double, _D, _D, _D, _D, _D, _D]
            L.or_step.argtypes = [_P, _D, _D, _D, _D, ctypes.c_double, _D]
            L.or_run.argtypes = [_P, _D, _D, _D, _D, ctypes.c_double, ctypes.c_long]
            L.or_run.restype = ctypes.c_long
            L.or_run_tangent.argtypes = [_P, _D, _D, _D, _D, _D, _D, _D, ctypes.c_double,
                                         ctypes.c_long]
            L.or_run_tangent.restype = ctypes.c_long
            L.or_flops_per_point_step.argtypes = [_P, _D, _D, _D]
            L.or_flops_per_point_step.restype = ctypes.c_double
            L.or_tangent_flops_per_point_step.argtypes = [_P, _D, _D, _D, _D, _D, _D]
            L.or_tangent_flops_per_point_step.restype = ctypes.c_double
            _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _arr(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None:
        assert a.size == n
    return a


# Paper defaults (Sec. 3): CFL 0.6, gamma = d = {0.98, 0.01, 0.01}, eps = 1e-6.
def problem(eq, dim, nx, ny=1, x0=0.0, x1=1.0, y0=0.0, y1=1.0, gas_gamma=1.4,
            bc=(BC_PERIODIC,) * 4, inflow=(0, 0, 0, 0), pre=(0, 0, 0, 0),
            dmr_x0=1.0 / 6.0, dmr_speed=10.0, dmr_angle=np.pi / 3.0,
            lin_w=(0.98, 0.01, 0.01), lim_d=(0.98, 0.01, 0.01), eps=1e-6, cfl=0.6,
            dt_mode=0, dt_fixed=0.0, limiter=1, eig_avg=0, alpha_fixed=0.0,
            freeze_weights=0) -> Problem:
    p = Problem()
    p.eq, p.dim, p.nx, p.ny = eq, dim, nx, (ny if dim == 2 else 1)
    p.x0, p.x1, p.y0, p.y1 = x0, x1, y0, y1
    p.gas_gamma = gas_gamma
    p.bc[:] = list(bc) + [BC_PERIODIC] * (4 - len(bc))
    p.inflow[:] = list(inflow) + [0.0] * (4 - len(inflow))
    p.pre[:] = list(pre) + [0.0] * (4 - len(pre))
    p.dmr_x0, p.dmr_speed, p.dmr_angle = dmr_x0, dmr_speed, dmr_angle
    p.lin_w[:] = lin_w
    p.lim_d[:] = lim_d
    p.eps, p.cfl, p.dt_mode, p.dt_fixed = eps, cfl, dt_mode, dt_fixed
    p.limiter, p.eig_avg = limiter, eig_avg
    p.alpha_fixed = alpha_fixed
    p.freeze_weights = int(freeze_weights)
    return p


def ncomp(p: Problem) -> int:
    return _load().or_ncomp(ctypes.byref(p))


def _shape(p):
    m = ncomp(p)
    return (m, p.nx) if p.dim == 1 else (m, p.ny, p.nx)


_FACE_KEYS = ("fhat", "hhat", "p0", "p1", "p2", "dp0", "beta0", "beta1", "beta2",
              "tau", "omega0", "omega1", "omega2")
_LIM_KEYS = ("vt", "dq0", "dq1", "dq2", "beta0", "beta1", "beta2", "tau",
             "lambda0", "lambda1", "lambda2")


def hweno_face(side, f, h, dx, lin_w=(0.98, 0.01, 0.01), eps=1e-6):
    """One-interface HWENO reconstruction (Sec. 2.1). side 0: "+" flux from
    (f, h) at i-1, i, i+1; side 1: "-" flux from (f, h) at i, i+1, i+2."""
    out = np.zeros(13)
    f, h, g = _arr(f, 3), _arr(h, 3), _arr(lin_w, 3)
    _load().or_hweno_face(side, _ptr(f), _ptr(h), dx, _ptr(g), eps, _ptr(out))
    return dict(zip(_FACE_KEYS, out))


def limiter(um, u0, up, vm, vp, dx, lim_d=(0.98, 0.01, 0.01), eps=1e-6):
    """HWENO limiter for the derivative at x_i (Sec. 2.2)."""
    out = np.zeros(11)
    d = _arr(lim_d, 3)
    _load().or_limiter(um, u0, up, vm, vp, dx, _ptr(d), eps, _ptr(out))
    return dict(zip(_LIM_KEYS, out))


def flux(p, direction, U):
    U = _arr(U)
    F = np.zeros_like(U)
    _load().or_flux(ctypes.byref(p), direction, _ptr(U), _ptr(F))
    return F


def jvp(p, direction, U, D):
    U, D = _arr(U), _arr(D)
    out = np.zeros_like(U)
    _load().or_jvp(ctypes.byref(p), direction, _ptr(U), _ptr(D), _ptr(out))
    return out


def wave_speed(p, direction, U):
    return _load().or_wave_speed(ctypes.byref(p), direction, _ptr(_arr(U)))


def eigen(p, direction, UL, UR=None):
    """(R, L, lambda) of the flux Jacobian at the average of UL, UR."""
    m = ncomp(p)
    Rm, Lm, lam = np.zeros((m, m)), np.zeros((m, m)), np.zeros(m)
    _load().or_eigen(ctypes.byref(p), direction, _ptr(_arr(UL)),
                     None if UR is None else _ptr(_arr(UR)), _ptr(Rm), _ptr(Lm), _ptr(lam))
    return Rm, Lm, lam


def rhs(p, U, V, W=None, t=0.0):
    """Spatial operators L^1, L^2 (, L^3), limited derivatives and alpha."""
    shp = _shape(p)
    U, V = _arr(U).reshape(shp), _arr(V).reshape(shp)
    L1, L2, Vt = np.zeros(shp), np.zeros(shp), np.zeros(shp)
    if p.dim == 1:
        al = np.zeros(1)
        _load().or_rhs_1d(ctypes.byref(p), _ptr(U), _ptr(V), t, _ptr(L1), _ptr(L2),
                          _ptr(Vt), _ptr(al))
        return dict(L1=L1, L2=L2, Vt=Vt, alpha=al)
    W = _arr(W).reshape(shp)
    L3, Wt, al = np.zeros(shp), np.zeros(shp), np.zeros(2)
    _load().or_rhs_2d(ctypes.byref(p), _ptr(U), _ptr(V), _ptr(W), t, _ptr(L1), _ptr(L2),
                      _ptr(L3), _ptr(Vt), _ptr(Wt), _ptr(al))
    return dict(L1=L1, L2=L2, L3=L3, Vt=Vt, Wt=Wt, alpha=al)


def step(p, U, V, W=None, t=0.0, t_end=np.inf):
    """One SSP-RK3 step on copies; returns (U, V, W, t, dt)."""
    shp = _shape(p)
    U, V = _arr(U).reshape(shp).copy(), _arr(V).reshape(shp).copy()
    W = _arr(W).reshape(shp).copy() if p.dim == 2 else None
    tt, dt = np.array([t], dtype=np.float64), np.zeros(1)
    _load().or_step(ctypes.byref(p), _ptr(U), _ptr(V), _ptr(W), _ptr(tt), t_end, _ptr(dt))
    return U, V, W, float(tt[0]), float(dt[0])


def run(p, U, V, W=None, t=0.0, t_end=1.0, max_steps=1 << 40):
    """SSP-RK3 steps until t_end (or max_steps); returns (U, V, W, t, steps)."""
    shp = _shape(p)
    U, V = _arr(U).reshape(shp).copy(), _arr(V).reshape(shp).copy()
    W = _arr(W).reshape(shp).copy() if p.dim == 2 else None
    tt = np.array([t], dtype=np.float64)
    k = _load().or_run(ctypes.byref(p), _ptr(U), _ptr(V), _ptr(W), _ptr(tt), t_end, max_steps)
    return U, V, W, float(tt[0]), int(k)


def run_tangent(p, U, V, W, dU, dV, dW=None, t=0.0, t_end=1.0, max_steps=1 << 40):
    """Forward-mode derivative of a run (dual numbers): returns
    (U, V, W, dU, dV, dW, t, steps) with alpha frozen in every stage (its
    state dependence is not differentiated) and the run's own time steps."""
    shp = _shape(p)
    U, V = _arr(U).reshape(shp).copy(), _arr(V).reshape(shp).copy()
    dU, dV = _arr(dU).reshape(shp).copy(), _arr(dV).reshape(shp).copy()
    two = p.dim == 2
    W = _arr(W).reshape(shp).copy() if two else None
    dW = _arr(dW).reshape(shp).copy() if two else None
    tt = np.array([t], dtype=np.float64)
    k = _load().or_run_tangent(ctypes.byref(p), _ptr(U), _ptr(V), _ptr(W), _ptr(dU), _ptr(dV),
                               _ptr(dW), _ptr(tt), t_end, max_steps)
    return U, V, W, dU, dV, dW, float(tt[0]), int(k)


def flops_per_point_step(p, U, V, W=None) -> float:
    """Algorithmic operations per grid point of one SSP-RK3 step, counted on
    the scheme as the oracle writes it (+ - * / sqrt count one each)."""
    shp = _shape(p)
    U, V = _arr(U).reshape(shp), _arr(V).reshape(shp)
    W = _arr(W).reshape(shp) if p.dim == 2 else None
    return _load().or_flops_per_point_step(ctypes.byref(p), _ptr(U), _ptr(V), _ptr(W))


def bl_alpha01():
    """max |f'(u)| over u in [0, 1] of the Buckley-Leverett flux (reading R15)."""
    return _load().or_bl_alpha01()


def hweno_face_tangent(side, f, h, df, dh, dx, lin_w=(0.98, 0.01, 0.01), eps=1e-6, frozen=False):
    """(d f-hat, d h-hat) of one face along (df, dh) (forward mode), with the
    nonlinear weights frozen or differentiated."""
    out = np.zeros(2)
    _load().or_hweno_face_tangent(side, _ptr(_arr(f, 3)), _ptr(_arr(h, 3)), _ptr(_arr(df, 3)),
                                  _ptr(_arr(dh, 3)), dx, _ptr(_arr(lin_w, 3)), eps, int(frozen),
                                  _ptr(out))
    return out


def limiter_tangent(um, u0, up, vm, vp, direction, dx, lim_d=(0.98, 0.01, 0.01), eps=1e-6,
                    frozen=False):
    """d v-tilde of the limiter along `direction` (5 values)."""
    return _load().or_limiter_tangent(um, u0, up, vm, vp, _ptr(_arr(direction, 5)), dx,
                                      _ptr(_arr(lim_d, 3)), eps, int(frozen))


def tangent_flops_per_point_step(p, U, V, W, dU, dV, dW=None) -> float:
    """Operations per grid point of one forward-mode (dual-number) step,
    values and tangents together (the work of one Jacobian-vector product of
    the step; the wave speeds frozen as in run_tangent)."""
    shp = _shape(p)
    U, V = _arr(U).reshape(shp), _arr(V).reshape(shp)
    dU, dV = _arr(dU).reshape(shp), _arr(dV).reshape(shp)
    W = _arr(W).reshape(shp) if p.dim == 2 else None
    dW = _arr(dW).reshape(shp) if p.dim == 2 else None
    return _load().or_tangent_flops_per_point_step(ctypes.byref(p), _ptr(U), _ptr(V), _ptr(W),
                                                   _ptr(dU), _ptr(dV), _ptr(dW))
