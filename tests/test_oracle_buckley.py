"""Pins of the oracle's Buckley-Leverett equation (Example 3.4): the flux and
its derivative against symbolic differentiation, alpha (reading R15) against
brute force and the cubic's root, the exact entropy solution's tangency
points against a symbolic solve, and the oracle's convergence to that exact
solution at T = 0.4."""
import numpy as np
import pytest

import oracle as O
from oracle import exact as E
from paper_2207_05258_gb300 import workloads as W
from _util import oracle_problem

sympy = pytest.importorskip("sympy")


def _p(n=8, **kw):
    return O.problem(O.EQ_BUCKLEY, 1, n, x0=-1.0, x1=1.0, **kw)


def test_flux_and_jvp_against_symbolic_derivative():
    u = sympy.Symbol("u")
    f = 4 * u ** 2 / (4 * u ** 2 + (1 - u) ** 2)
    fs = sympy.lambdify(u, f)
    dfs = sympy.lambdify(u, sympy.diff(f, u))
    P = _p()
    rng = np.random.default_rng(1)
    for x in np.concatenate([rng.uniform(-0.5, 1.5, 40), [0.0, 1.0, 0.3]]):
        assert abs(O.flux(P, 0, [x])[0] - fs(x)) <= 1e-15 * max(1, abs(fs(x)))
        d = rng.standard_normal()
        assert abs(O.jvp(P, 0, [x], [d])[0] - dfs(x) * d) <= 1e-14 * max(1, abs(dfs(x) * d))


def test_alpha_over_admissible_states():
    a = O.bl_alpha01()
    # brute force over [0, 1]
    uu = np.linspace(0.0, 1.0, 2_000_001)
    brute = np.max(np.abs(E.bl_df(uu)))
    assert abs(a - brute) <= 1e-11
    # the interior maximum of f' sits at the root in (0, 1) of d f'/du = 0
    u = sympy.Symbol("u")
    f = 4 * u ** 2 / (4 * u ** 2 + (1 - u) ** 2)
    crit = [complex(r).real for r in sympy.Poly(sympy.numer(sympy.together(
        sympy.diff(f, u, 2))), u).nroots(n=30) if abs(complex(r).imag) < 1e-20]
    inside = [r for r in crit if 0 < r < 1]
    assert len(inside) == 1
    assert abs(a - E.bl_df(inside[0])) <= 1e-14
    # the per-point wave speed never falls below it (reading R15)
    P = _p()
    for x in (-3.0, -0.24, 0.0, 0.287, 1.0, 1.45, 4.0):
        assert O.wave_speed(P, 0, [x]) == pytest.approx(max(a, abs(E.bl_df(x))), rel=1e-15)


def test_exact_solution_tangency_points():
    u = sympy.Symbol("u", positive=True)
    f = 4 * u ** 2 / (4 * u ** 2 + (1 - u) ** 2)
    df = sympy.diff(f, u)
    ua = [float(r) for r in sympy.solve(sympy.simplify(df * u - f), u) if 0 < float(r) < 1]
    ub = [float(r) for r in sympy.solve(sympy.simplify(df * (1 - u) - (1 - f)), u)
          if 0 < float(r) < 1]
    assert ua and abs(ua[0] - 1 / np.sqrt(5)) < 1e-15
    assert abs(min(ub) - (1 - 2 / np.sqrt(5))) < 1e-15
    # the exact profile at T: monotone pieces, the fans invert f'
    x = np.linspace(-1, 1, 2001)
    ue = E.buckley_leverett_exact(x, 0.4)
    fan = (x > 0.001) & (x < 0.4 * E.bl_f(ua[0]) / ua[0] - 0.001)
    assert np.allclose(E.bl_df(ue[fan]), x[fan] / 0.4, rtol=0, atol=1e-12)
    assert np.all(np.diff(ue[fan]) <= 0)


def test_oracle_converges_to_the_entropy_solution():
    errs = []
    for n in (80, 160, 320):
        w = W.buckley_leverett(n)
        U, V, _, t, k = O.run(oracle_problem(w), w.U, w.V, None, 0.0, w.t_end)
        assert t == w.t_end
        x = W.centers(-1.0, 1.0, n)
        errs.append(float(np.mean(np.abs(U.ravel() - E.buckley_leverett_exact(x, w.t_end)))))
    assert errs[0] < 0.03 and errs[1] < errs[0] and errs[2] < errs[1], errs
    assert errs[2] < 0.6 * errs[0], errs


def test_periodic_conservation_and_bounds():
    n = 64
    x = W.centers(-1.0, 1.0, n)
    U = 0.5 + 0.4 * np.sin(np.pi * x)
    V = 0.4 * np.pi * np.cos(np.pi * x)
    P = O.problem(O.EQ_BUCKLEY, 1, n, x0=-1.0, x1=1.0)
    U1, _, _, _, k = O.run(P, U, V, None, 0.0, 0.3)
    assert abs(U1.sum() - U.sum()) <= 1e-12 * n
    assert U1.min() > -1e-6 and U1.max() < 1 + 1e-6
