"""The oracle against the paper's printed accuracy tables (Tables 1-5,
Examples 3.1, 3.2, 3.8, 3.9; fixtures under tests/golden/ with their
citations). Errors are the grid-average L1 and the max norm of u (density for
Euler) at T against the exact solution; dt = CFL dx^{5/3}/alpha (the reading
under which the printed magnitudes are reproduced). The coarse-grid sizes
run in seconds; the fifth order and the magnitudes are both checked."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import exact
from paper_2207_05258_gb300 import workloads as W
from _util import load_table, norms, oracle_problem

# |log(ours / printed)| bound. On the grids with N <= 20 a run takes 4-20
# steps and the printed errors depend on time-step details the paper does not
# state (the 1D Burgers rows N = 10, 20 move by 2x between plausible dt
# rules), so only a factor 2.5 is asserted there; from N = 40 on the printed
# values are matched within 15%.
def close(ours, printed, n):
    return abs(math.log(ours / printed)) < math.log(2.5 if n <= 20 else 1.15)


def run_burgers1d(n):
    w = W.burgers1d_sine(n, t_end=0.5 / math.pi, dt_mode="accuracy")
    U, _, _, t, _ = O.run(oracle_problem(w), w.U, w.V, None, 0.0, w.t_end)
    x = W.centers(0, 2, n)
    ue = exact.burgers_characteristics(x, w.t_end, lambda s: 0.5 + np.sin(np.pi * s),
                                       lambda s: np.pi * np.cos(np.pi * s))
    return norms(U[0] - ue)


def run_euler1d(n, **kw):
    w = W.euler1d_smooth(n)
    U, _, _, t, _ = O.run(oracle_problem(w, **kw), w.U, w.V, None, 0.0, w.t_end)
    x = W.centers(0, 2, n)
    return norms(U[0] - (1 + 0.2 * np.sin(np.pi * (x - w.t_end))))


def run_burgers2d(n):
    w = W.burgers2d_sine(n)
    U, _, _, t, _ = O.run(oracle_problem(w), w.U, w.V, w.W, 0.0, w.t_end)
    x = W.centers(0, 4, n)
    X, Y = np.meshgrid(x, x)
    ue = exact.burgers_characteristics(X + Y, w.t_end, lambda s: 0.5 + np.sin(np.pi * s / 2),
                                       lambda s: 0.5 * np.pi * np.cos(np.pi * s / 2), speed=2.0)
    return norms(U[0] - ue)


def run_euler2d(n, **kw):
    w = W.euler2d_smooth(n, u=1.0, v=1.0)
    U, _, _, t, _ = O.run(oracle_problem(w, **kw), w.U, w.V, w.W, 0.0, w.t_end)
    x = W.centers(0, 2, n)
    X, Y = np.meshgrid(x, x)
    return norms(U[0] - (1 + 0.2 * np.sin(np.pi * (X + Y - 2 * w.t_end))))


CASES = [
    ("table1_burgers1d.txt", run_burgers1d, (10, 20, 40, 80, 160)),
    ("table2_euler1d.txt", run_euler1d, (10, 20, 40, 80)),
    ("table3_burgers2d.txt", run_burgers2d, (10, 20, 40)),
    ("table4_euler2d.txt", run_euler2d, (10, 20)),
]


@pytest.mark.parametrize("table,fn,sizes", CASES, ids=[c[0][:-4] for c in CASES])
def test_matches_printed_table(table, fn, sizes):
    ref = load_table(table)
    got = {n: fn(n) for n in sizes}
    for n in sizes:
        l1, li = got[n]
        assert close(l1, ref[n][0], n), (n, l1, ref[n][0])
        assert close(li, ref[n][1], n), (n, li, ref[n][1])
    big = [n for n in sizes if n >= 40]
    for a, b in zip(big, big[1:]):
        order = math.log2(got[a][0] / got[b][0])
        assert order > 4.5, (a, b, order)


def test_without_limiter_matches_table5_coarse():
    """Table 5: the scheme without the limiter on the coarse grids."""
    ref = load_table("table5_euler2d_nolimiter.txt")
    for n in (10, 20):
        l1, li = run_euler2d(n, limiter=0)
        assert close(l1, ref[n][0], n), (n, l1, ref[n][0])
        assert close(li, ref[n][1], n), (n, li, ref[n][1])
