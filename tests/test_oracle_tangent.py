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


# ---------------------------------------------------------------------------
# Frozen-weights derivative (the option of the adjoint that holds the
# nonlinear weights at their forward values)
# ---------------------------------------------------------------------------
def _face_closed_form(side, f, h, df, dh, dx, g, eps):
    """d f-hat with the weights held: sum_l omega_l d(candidate_l), the
    candidates being linear in the data (their values come from or_hweno_face
    at the perturbation itself, since p_l(d) = d p_l)."""
    o = O.hweno_face(side, f, h, dx, g, eps)
    z = O.hweno_face(side, df, dh, dx, g, eps)  # p_0, p_1, p_2 of the direction
    w = (o["omega0"], o["omega1"], o["omega2"])
    p = (z["p0"], z["p1"], z["p2"])
    return w[0] * (p[0] / g[0] - g[1] / g[0] * p[1] - g[2] / g[0] * p[2]) + w[1] * p[1] + w[2] * p[2]


def test_face_tangent_frozen_weights_is_the_weighted_candidate_derivative():
    rng = np.random.default_rng(3)
    g = (0.98, 0.01, 0.01)
    for side in (0, 1):
        for _ in range(20):
            f, h = rng.standard_normal(3), rng.standard_normal(3)
            df, dh = rng.standard_normal(3), rng.standard_normal(3)
            dx = rng.uniform(0.01, 0.5)
            got = O.hweno_face_tangent(side, f, h, df, dh, dx, g, 1e-6, frozen=True)[0]
            want = _face_closed_form(side, f, h, df, dh, dx, g, 1e-6)
            assert abs(got - want) <= 1e-12 * (1 + abs(want)), (side, got, want)


def test_face_tangent_unfrozen_against_central_differences():
    rng = np.random.default_rng(4)
    g = (0.98, 0.01, 0.01)
    for side in (0, 1):
        for _ in range(10):
            f, h = rng.standard_normal(3), rng.standard_normal(3)
            df, dh = rng.standard_normal(3), rng.standard_normal(3)
            got = O.hweno_face_tangent(side, f, h, df, dh, 0.1, g, 1e-6)[0]
            e = 1e-6
            fd = (O.hweno_face(side, f + e * df, h + e * dh, 0.1, g, 1e-6)["fhat"] -
                  O.hweno_face(side, f - e * df, h - e * dh, 0.1, g, 1e-6)["fhat"]) / (2 * e)
            assert abs(got - fd) <= 1e-6 * (1 + abs(fd)), (got, fd)


def test_limiter_tangent_frozen_and_unfrozen():
    rng = np.random.default_rng(5)
    d = (0.98, 0.01, 0.01)
    for _ in range(20):
        x = rng.standard_normal(5)
        dirn = rng.standard_normal(5)
        dx = 0.1
        o = O.limiter(*x, dx, d, 1e-6)
        z = O.limiter(*dirn, dx, d, 1e-6)  # dq_l of the direction (linear)
        lam, dq = (o["lambda0"], o["lambda1"], o["lambda2"]), (z["dq0"], z["dq1"], z["dq2"])
        want = lam[0] * (dq[0] / d[0] - d[1] / d[0] * dq[1] - d[2] / d[0] * dq[2]) + \
            lam[1] * dq[1] + lam[2] * dq[2]
        got = O.limiter_tangent(*x, dirn, dx, d, 1e-6, frozen=True)
        assert abs(got - want) <= 1e-12 * (1 + abs(want))
        e = 1e-6
        fd = (O.limiter(*(x + e * dirn), dx, d, 1e-6)["vt"] -
              O.limiter(*(x - e * dirn), dx, d, 1e-6)["vt"]) / (2 * e)
        got_full = O.limiter_tangent(*x, dirn, dx, d, 1e-6)
        assert abs(got_full - fd) <= 1e-6 * (1 + abs(fd))
