"""Shocked runs of the oracle against what is known exactly: the exact
Riemann solver (Toro) for 1D Euler with outflow boundaries, the entropy
solution of the sine Burgers problem after breaking (Example 3.3), the
Rankine-Hugoniot post-shock state of the double Mach reflection set-up
(Example 3.11), positivity, and the Roe/mean eigenvector option."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import exact
from paper_2207_05258_gb300 import workloads as W
from _util import oracle_problem

G = 1.4


def riemann_l1(left, right, n, t_end=0.15, **kw):
    w = W.riemann1d(n, left, right, t_end=t_end)
    U, _, _, t, k = O.run(oracle_problem(w, **kw), w.U, w.V, None, 0.0, w.t_end)
    x = W.centers(0, 1, n)
    rho, u, p, _, _ = exact.riemann_exact(left, right, G, x, t_end)
    assert t == t_end
    return float(np.mean(np.abs(U[0] - rho))), U


@pytest.mark.parametrize("states", [
    ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1)),                      # Sod
    ((0.445, 0.698, 3.528), (0.5, 0.0, 0.571)),                # Lax (Example 3.5 states)
] + [W.riemann_batch(count=4, seed=7).meta["states"][k] for k in range(4)])
def test_riemann_against_exact_solution(states):
    left, right = states
    errs = []
    for n in (100, 200, 400):
        e, U = riemann_l1(left, right, n)
        errs.append(e)
        rho = U[0]
        m, E = U[1], U[2]
        p = (G - 1) * (E - 0.5 * m * m / rho)
        assert np.all(rho > 0) and np.all(p > 0)
    assert errs[1] < errs[0] and errs[2] < errs[1], errs
    assert errs[2] < 1.2e-2, errs


def test_exact_riemann_solver_sod_star_state():
    """Toro's Table 4.2 star values for Sod's test 1: p* = 0.30313, u* = 0.92745."""
    _, _, _, ps, us = exact.riemann_exact((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), G, [0.5], 0.1)
    assert abs(ps - 0.30313) < 1e-5 and abs(us - 0.92745) < 1e-5


def burgers_sine_entropy(x, t):
    """Entropy solution of u_t + (u^2/2)_x = 0, u0 = 0.5 + sin(pi x) on [0, 2]
    periodic, for t > 1/pi: in the frame moving at 1/2, w = u - 1/2 has w0 odd
    about 1 and a steady shock at 1; left of it w comes from the increasing
    branch xi in [0, xi_c] of xi + t sin(pi xi)."""
    xs = np.mod(x - 0.5 * t, 2.0)
    xi_c = math.acos(-1.0 / (math.pi * t)) / math.pi
    out = np.empty_like(xs)
    for k, y in enumerate(xs):
        s, yy = (1.0, y) if y < 1.0 else (-1.0, 2.0 - y)
        lo, hi = 0.0, xi_c
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if mid + t * math.sin(math.pi * mid) < yy:
                lo = mid
            else:
                hi = mid
        out[k] = 0.5 + s * math.sin(math.pi * 0.5 * (lo + hi))
    return out, 1.0 + 0.5 * t


def test_burgers_shock_example_3_3():
    n, T = 400, 1.5 / math.pi
    w = W.burgers1d_sine(n, t_end=T)
    U, _, _, t, k = O.run(oracle_problem(w), w.U, w.V, None, 0.0, T)
    x = W.centers(0, 2, n)
    ue, xs = burgers_sine_entropy(x, T)
    away = np.abs(x - xs) > 0.03
    assert np.max(np.abs(U[0][away] - ue[away])) < 2e-4
    jump = np.argmin(np.diff(U[0]))
    assert abs(0.5 * (x[jump] + x[jump + 1]) - xs) < 1.5 * (2.0 / n)
    # essentially non-oscillatory: overshoots stay below 0.25% of the range
    assert U[0].max() < 1.5 + 5e-3 and U[0].min() > -0.5 - 5e-3


def test_dmr_post_shock_state_is_rankine_hugoniot():
    rho2, p2, u2 = exact.normal_shock_post_state(10.0, 1.4, 1.0, G)
    assert abs(rho2 - W.DMR_POST[0]) < 1e-12 and abs(p2 - W.DMR_POST[3]) < 1e-12
    assert abs(math.hypot(W.DMR_POST[1], W.DMR_POST[2]) - u2) < 1e-12
    # the post-shock velocity is normal to the shock line at 60 degrees
    assert abs(W.DMR_POST[1] * math.cos(math.pi / 3) + W.DMR_POST[2] * math.sin(math.pi / 3)) < 1e-12


def test_dmr_short_run_positive():
    w = W.double_mach(64, 16, t_end=0.01)
    P = oracle_problem(w)
    U, V, Wd, t, k = O.run(P, w.U, w.V, w.W, 0.0, w.t_end)
    U = U.reshape(4, 16, 64)
    rho, E = U[0], U[3]
    p = (G - 1) * (E - 0.5 * (U[1] ** 2 + U[2] ** 2) / rho)
    assert t == w.t_end and k > 5
    assert np.all(np.isfinite(U)) and np.all(rho > 0) and np.all(p > 0)
    # far right, ahead of the shock, the gas is still at rest
    assert np.allclose(U[:, :, -8:], np.array(w.pre)[:, None, None], atol=1e-10)


def test_lax_example_against_exact_solution():
    """Example 3.5 (Lax problem) at T = 0.16: the L1 density error against the
    exact Riemann solution falls with N."""
    errs = []
    for n in (100, 200, 400):
        w = W.lax(n)
        U, _, _, t, _ = O.run(oracle_problem(w), w.U, w.V, None, 0.0, w.t_end)
        x = W.centers(-0.5, 0.5, n)
        rho = exact.riemann_exact((0.445, 0.698, 3.528), (0.5, 0.0, 0.571), G, x, w.t_end, x0=0.0)[0]
        errs.append(float(np.mean(np.abs(U[0] - rho))))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-2, errs


def test_blast_waves_stay_physical_and_conserve_mass():
    """Example 3.7 with reflective walls: mass is conserved exactly by the
    flux form with mirrored ghosts (zero mass flux through the walls)."""
    w = W.blast_waves(200, t_end=0.01)
    U, _, _, t, _ = O.run(oracle_problem(w), w.U, w.V, None, 0.0, w.t_end)
    rho, m, E = U
    p = (G - 1) * (E - 0.5 * m * m / rho)
    assert np.all(rho > 0) and np.all(p > 0)
    assert abs(rho.sum() - w.U.reshape(3, -1)[0].sum()) < 1e-12 * rho.sum()
