"""Pins of the oracle's forward-mode (dual-number) derivative, the reference
for the GPU adjoint. With a prescribed alpha and a fixed time step a step is
a smooth function of the state (away from the |.| kinks of tau), so the
dual tangent must equal central finite differences; the value part must
equal the plain run bit for bit; and the tangent is linear in the seed."""
import numpy as np
import pytest

import oracle as O
from paper_2207_05258_gb300 import workloads as W
from _util import oracle_problem


def fd(P, U, V, Wd, dU, dV, dWd, steps, eps):
    plus = O.run(P, U + eps * dU, V + eps * dV, None if Wd is None else Wd + eps * dWd, 0.0, 10.0,
                 max_steps=steps)
    minus = O.run(P, U - eps * dU, V - eps * dV, None if Wd is None else Wd - eps * dWd, 0.0,
                  10.0, max_steps=steps)
    return [(a - b) / (2 * eps) for a, b in zip(plus[:2], minus[:2])]


@pytest.mark.parametrize("case", ["burgers1d", "euler1d", "euler2d"])
def test_tangent_matches_finite_differences(case):
    rng = np.random.default_rng(3)
    if case == "burgers1d":
        w = W.burgers1d_sine(64)
        P = oracle_problem(w, dt_mode=2, dt_fixed=2e-3, alpha_fixed=1.6)
        U, V, Wd = w.U.reshape(1, -1), w.V.reshape(1, -1), None
    elif case == "euler1d":
        w = W.euler1d_smooth(48)
        P = oracle_problem(w, dt_mode=2, dt_fixed=4e-3, alpha_fixed=2.5)
        U, V, Wd = w.U.reshape(3, -1), w.V.reshape(3, -1), None
    else:
        w = W.euler2d_smooth(12, u=0.4, v=-0.2)
        P = oracle_problem(w, dt_mode=2, dt_fixed=8e-3, alpha_fixed=2.0)
        U, V, Wd = (a.reshape(4, 12, 12) for a in (w.U, w.V, w.W))
    dU, dV = rng.standard_normal(U.shape) * 1e-2, rng.standard_normal(V.shape) * 1e-1
    dWd = rng.standard_normal(U.shape) * 1e-1 if Wd is not None else None
    steps = 3
    out = O.run_tangent(P, U, V, Wd, dU, dV, dWd, 0.0, 10.0, max_steps=steps)
    plain = O.run(P, U, V, Wd, 0.0, 10.0, max_steps=steps)
    assert np.array_equal(out[0], plain[0]) and np.array_equal(out[1], plain[1])
    gU, gV = fd(P, U, V, Wd, dU, dV, dWd, steps, 1e-6)
    assert np.max(np.abs(out[3] - gU)) <= 1e-6 * max(np.max(np.abs(gU)), 1e-3)
    assert np.max(np.abs(out[4] - gV)) <= 1e-6 * max(np.max(np.abs(gV)), 1e-3)


def test_tangent_is_linear_in_the_seed():
    w = W.burgers1d_sine(40)
    P = oracle_problem(w)
    rng = np.random.default_rng(4)
    U, V = w.U.reshape(1, -1), w.V.reshape(1, -1)
    a = rng.standard_normal(U.shape), rng.standard_normal(V.shape)
    b = rng.standard_normal(U.shape), rng.standard_normal(V.shape)
    ta = O.run_tangent(P, U, V, None, *a, None, 0.0, 0.2)
    tb = O.run_tangent(P, U, V, None, *b, None, 0.0, 0.2)
    tc = O.run_tangent(P, U, V, None, 2 * a[0] - b[0], 2 * a[1] - b[1], None, 0.0, 0.2)
    assert np.allclose(tc[3], 2 * ta[3] - tb[3], rtol=1e-12, atol=1e-12)
    assert np.allclose(tc[4], 2 * ta[4] - tb[4], rtol=1e-12, atol=1e-10)
