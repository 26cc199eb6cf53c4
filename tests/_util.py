"""Shared test helpers: map a workload onto the oracle's problem record and
error norms. Error norms (paper, Sec. 3): L1 = grid average of |e|, Linf = max."""
import os

import numpy as np

import oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

BC = dict(periodic=O.BC_PERIODIC, outflow=O.BC_OUTFLOW, reflective=O.BC_REFLECTIVE,
          inflow=O.BC_INFLOW, dmr_bottom=O.BC_DMR_BOTTOM, dmr_top=O.BC_DMR_TOP)


def oracle_problem(w, nx=None, **kw):
    """Oracle problem record for workload `w` (instance size `nx` in a batch)."""
    args = dict(dt_mode=1 if w.dt_mode == "accuracy" else 0)
    args.update(kw)
    eq = dict(burgers=O.EQ_BURGERS, euler=O.EQ_EULER, buckley=O.EQ_BUCKLEY)[w.equation]
    return O.problem(eq, w.dim,
                     nx if nx is not None else w.nx[0], w.ny, w.x0, w.x1, w.y0, w.y1,
                     w.gas_gamma, tuple(BC[b] for b in w.bc), w.inflow, w.pre, w.dmr_x0,
                     w.dmr_speed, w.dmr_angle, **args)


def shape(w):
    return (w.m, w.nx[0]) if w.dim == 1 else (w.m, w.ny, w.nx[0])


def norms(e):
    e = np.abs(np.asarray(e))
    return float(e.mean()), float(e.max())


def load_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            p = line.split()
            rows.append((int(p[0]), float(p[1]), float(p[3])))
    return {n: (l1, li) for n, l1, li in rows}


def header_functions():
    """Names of the functions declared in include/hweno.h."""
    import re
    root = os.path.dirname(GOLDEN[:-len("/golden")])
    src = open(os.path.join(root, "include", "hweno.h")).read()
    return sorted(set(re.findall(r"^(?:int|long long|const char\*)\s+(hweno_\w+)\s*\(", src, re.M)))


def scales_1d(w, U, k=None):
    """(U_scale, F_scale) of one 1D instance: max|U| and max over points of
    |f(U)| + alpha |U| (the size of the split fluxes)."""
    import oracle as O
    P = oracle_problem(w, nx=U.shape[1])
    us = float(np.max(np.abs(U)))
    al = max(O.wave_speed(P, 0, U[:, i]) for i in range(U.shape[1]))
    fs = max(float(np.max(np.abs(O.flux(P, 0, U[:, i])))) for i in range(U.shape[1]))
    return us, fs + al * us


def max_err(a, b):
    return float(np.max(np.abs(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64))))
