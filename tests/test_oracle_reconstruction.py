"""Pins of the oracle's per-interface reconstruction (Sec. 2.1) and limiter
(Sec. 2.2) against brute force: the Hermite conditions of Eq. HWEp0/HWEp12
and of the limiter's q_0, q_1, q_2 are solved as linear systems, and the
smoothness indicators of Eq. GHYZ / GHYZ-q are integrated by Gauss-Legendre
quadrature (exact for these polynomial integrands). Work is in the scaled
coordinate xi = (x - x_i)/dx, so cell I_{i+l} is [l - 1/2, l + 1/2]."""
import zlib

import numpy as np
import pytest

import oracle as O

GL_X, GL_W = np.polynomial.legendre.leggauss(10)


def cell_avg_monomial(k, a, b):
    return (b ** (k + 1) - a ** (k + 1)) / ((k + 1) * (b - a))


def poly_eval(c, x, der=0):
    return np.polynomial.polynomial.polyval(x, np.polynomial.polynomial.polyder(c, der) if der else c)


def hermite_avg_poly(deg, cells_f, cells_h, f, h):
    """Polynomial of degree `deg` whose cell averages over [l-1/2, l+1/2]
    are f (l in cells_f) and whose derivative averages are h (l in cells_h);
    h is the scaled derivative dx * h."""
    rows, rhs = [], []
    for l, val in zip(cells_f, f):
        rows.append([cell_avg_monomial(k, l - 0.5, l + 0.5) for k in range(deg + 1)])
        rhs.append(val)
    for l, val in zip(cells_h, h):
        # average of p' over the cell = p(b) - p(a) (unit cell width)
        rows.append([(l + 0.5) ** k - (l - 0.5) ** k for k in range(deg + 1)])
        rhs.append(val)
    return np.linalg.solve(np.array(rows, dtype=np.float64), np.array(rhs))


def smoothness(c, center=0.0):
    """sum_{a>=1} int_{center-1/2}^{center+1/2} (d^a p / dxi^a)^2 dxi."""
    deg = len(c) - 1
    xs = center + 0.5 * GL_X
    total = 0.0
    for a in range(1, deg + 1):
        total += 0.5 * np.sum(GL_W * poly_eval(c, xs, a) ** 2)
    return total


def brute_face(f, h, dx, g, eps, side):
    """Brute-force f-hat, h-hat and intermediates at x_{i+1/2}.
    side 0: stencil {i-1, i, i+1}, target cell I_i, interface at xi = +1/2.
    side 1 (mirror): stencil {i, i+1, i+2}, target cell I_{i+1} centred at 0,
    interface at xi = -1/2; the small stencils are the mirror images of T1, T2:
    {i+2, i+1} and {i, i+1}."""
    H = dx * np.asarray(h)
    if side == 0:
        c0 = hermite_avg_poly(5, [-1, 0, 1], [-1, 0, 1], f, H)
        c1 = hermite_avg_poly(2, [-1, 0], [0], [f[0], f[1]], [H[1]])
        c2 = hermite_avg_poly(2, [0, 1], [0], [f[1], f[2]], [H[1]])
        xe = 0.5
    else:
        c0 = hermite_avg_poly(5, [-1, 0, 1], [-1, 0, 1], f, H)
        c1 = hermite_avg_poly(2, [1, 0], [0], [f[2], f[1]], [H[1]])
        c2 = hermite_avg_poly(2, [-1, 0], [0], [f[0], f[1]], [H[1]])
        xe = -0.5
    p = [poly_eval(c, xe) for c in (c0, c1, c2)]
    dp0 = poly_eval(c0, xe, 1) / dx
    beta = [smoothness(c) for c in (c0, c1, c2)]
    tau = 0.25 * (abs(beta[0] - beta[1]) + abs(beta[0] - beta[2])) ** 2
    wb = [g[l] * (1.0 + tau / (beta[l] + eps)) for l in range(3)]
    om = [w / sum(wb) for w in wb]
    fhat = om[0] * (p[0] / g[0] - g[1] / g[0] * p[1] - g[2] / g[0] * p[2]) + om[1] * p[1] + om[2] * p[2]
    return dict(fhat=fhat, hhat=dp0, p0=p[0], p1=p[1], p2=p[2], beta0=beta[0], beta1=beta[1],
                beta2=beta[2], tau=tau, omega0=om[0], omega1=om[1], omega2=om[2])


def rel(a, b, scale=1.0):
    return abs(a - b) / max(abs(b), scale)


CASES = [
    ("smooth", lambda r: (1.0 + 0.1 * r.standard_normal(3), 0.3 * r.standard_normal(3))),
    ("rough", lambda r: (r.standard_normal(3), 5.0 * r.standard_normal(3))),
    ("jump", lambda r: (np.array([1.0, 1.0, 0.1]) + 0.01 * r.standard_normal(3), r.standard_normal(3))),
]


@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("g", [(0.98, 0.01, 0.01), (0.9, 0.06, 0.04), (1 / 3, 1 / 3, 1 / 3)])
def test_face_matches_brute_force(side, case, g):
    rng = np.random.default_rng(zlib.crc32(repr((side, case[0], g)).encode()))
    for dx in (0.5, 0.05, 0.002):
        for _ in range(8):
            f, h = case[1](rng)
            got = O.hweno_face(side, f, h, dx, g, 1e-6)
            ref = brute_face(f, h, dx, g, 1e-6, side)
            fs = max(1.0, np.max(np.abs(f)))
            for k in ("p0", "p1", "p2"):
                assert rel(got[k], ref[k], fs) < 1e-12, (k, got[k], ref[k])
            assert rel(got["hhat"], ref["hhat"], fs / dx) < 1e-11
            bs = max(ref["beta0"], ref["beta1"], ref["beta2"], 1e-30)
            for k in ("beta0", "beta1", "beta2"):
                assert abs(got[k] - ref[k]) <= 1e-11 * bs, (k, got[k], ref[k])
            for k in ("omega0", "omega1", "omega2"):
                assert abs(got[k] - ref[k]) < 1e-9, (k, got[k], ref[k])
            assert rel(got["fhat"], ref["fhat"], fs) < 1e-9


def test_beta2_uses_right_neighbour():
    """Eq. GHYZP prints f_{i-1} in beta_2; the defining integral gives f_{i+1}.
    Data with f_{i-1} != f_{i+1} separate the two readings."""
    f, h, dx = np.array([0.0, 1.0, 3.0]), np.array([0.2, 0.5, -0.1]), 0.1
    got = O.hweno_face(0, f, h, dx)
    H0 = dx * h[1]
    printed = H0 ** 2 + 13.0 / 3.0 * (H0 + f[1] - f[0]) ** 2
    brute = brute_face(f, h, dx, (0.98, 0.01, 0.01), 1e-6, 0)["beta2"]
    assert abs(got["beta2"] - brute) < 1e-12 * brute
    assert abs(got["beta2"] - printed) > 1.0


def test_quintic_exactness():
    """p_0 reproduces any quintic: with exact cell averages of phi and phi',
    p_0(x_{i+1/2}) = phi(x_{i+1/2}) and p_0'(x_{i+1/2}) = phi'(x_{i+1/2})."""
    rng = np.random.default_rng(5)
    for dx in (1.0, 0.1, 0.01):
        for _ in range(10):
            c = rng.standard_normal(6)
            P = np.polynomial.Polynomial(c)
            iP, dP = P.integ(), P.deriv()
            xs = np.array([-1.0, 0.0, 1.0]) * dx
            f = (iP(xs + dx / 2) - iP(xs - dx / 2)) / dx
            h = (P(xs + dx / 2) - P(xs - dx / 2)) / dx
            got = O.hweno_face(0, f, h, dx)
            s = np.max(np.abs(c)) * 4
            assert abs(got["p0"] - P(dx / 2)) < 1e-13 * s
            assert abs(got["hhat"] - dP(dx / 2)) < 1e-12 * s / dx
            # mirror: stencil {i, i+1, i+2} = xs + dx, interface x_{i+1/2} = dx/2
            f2 = (iP(xs + 1.5 * dx) - iP(xs + 0.5 * dx)) / dx
            h2 = (P(xs + 1.5 * dx) - P(xs + 0.5 * dx)) / dx
            got2 = O.hweno_face(1, f2, h2, dx)
            assert abs(got2["p0"] - P(dx / 2)) < 1e-13 * s
            assert abs(got2["hhat"] - dP(dx / 2)) < 1e-12 * s / dx


def test_quadratic_exactness_any_weights():
    """For quadratic phi, p_0 = p_1 = p_2 = phi(x_{i+1/2}) so the nonlinear
    combination returns phi(x_{i+1/2}) whatever the weights."""
    rng = np.random.default_rng(6)
    for g in [(0.98, 0.01, 0.01), (0.2, 0.5, 0.3)]:
        for _ in range(20):
            c = rng.standard_normal(3) * 10
            dx = 10 ** rng.uniform(-3, 0)
            P = np.polynomial.Polynomial(c)
            iP = P.integ()
            for side, xs, xe in ((0, np.array([-1, 0, 1]) * dx, dx / 2),
                                 (1, np.array([0, 1, 2]) * dx, dx / 2)):
                f = (iP(xs + dx / 2) - iP(xs - dx / 2)) / dx
                h = (P(xs + dx / 2) - P(xs - dx / 2)) / dx
                got = O.hweno_face(side, f, h, dx, g)
                assert abs(got["fhat"] - P(xe)) < 1e-11 * (1 + abs(P(xe))) * 10


def test_weights_tend_to_linear_on_smooth_data():
    """Smooth data: tau = O(dx^10) against beta = O(dx^2), so omega -> gamma
    as dx -> 0 (the nonlinear weights keep the fifth order)."""
    errs, taus = [], []
    for dx in (0.4, 0.2, 0.1, 0.05, 0.025):
        xs = np.array([-1.0, 0.0, 1.0]) * dx + 0.3
        f = (-np.cos(xs + dx / 2) + np.cos(xs - dx / 2)) / dx
        h = (np.sin(xs + dx / 2) - np.sin(xs - dx / 2)) / dx
        got = O.hweno_face(0, f, h, dx)
        errs.append(abs(got["omega0"] - 0.98))
        taus.append(got["tau"])
    assert all(b <= a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-14
    assert all(a / b > 2.0 ** 9 for a, b in zip(taus, taus[1:]))


def brute_limiter(um, u0, up, vm, vp, dx, d, eps):
    # q0: quartic with q(-1)=um, q(0)=u0, q(1)=up, q'(-1)=dx vm, q'(1)=dx vp
    rows = [[(-1.0) ** k for k in range(5)], [1.0 if k == 0 else 0.0 for k in range(5)],
            [1.0] * 5, [k * (-1.0) ** (k - 1) if k else 0.0 for k in range(5)],
            [float(k) for k in range(5)]]
    c0 = np.linalg.solve(np.array(rows), np.array([um, u0, up, dx * vm, dx * vp]))
    c1 = np.array([u0, u0 - um])
    c2 = np.array([u0, up - u0])
    dq = [poly_eval(c, 0.0, 1) / dx for c in (c0, c1, c2)]
    beta = [smoothness(c) for c in (c0, c1, c2)]
    tau = 0.25 * (abs(beta[0] - beta[1]) + abs(beta[0] - beta[2])) ** 2
    lb = [d[l] * (1.0 + tau / (beta[l] + eps)) for l in range(3)]
    lam = [x / sum(lb) for x in lb]
    vt = lam[0] * (dq[0] / d[0] - d[1] / d[0] * dq[1] - d[2] / d[0] * dq[2]) + lam[1] * dq[1] + lam[2] * dq[2]
    return dict(vt=vt, dq0=dq[0], dq1=dq[1], dq2=dq[2], beta0=beta[0], beta1=beta[1],
                beta2=beta[2], tau=tau, lambda0=lam[0], lambda1=lam[1], lambda2=lam[2])


@pytest.mark.parametrize("d", [(0.98, 0.01, 0.01), (0.5, 0.3, 0.2)])
def test_limiter_matches_brute_force(d):
    rng = np.random.default_rng(7)
    for dx in (0.5, 0.05, 0.001):
        for scale in (0.01, 1.0, 30.0):
            for _ in range(8):
                u = 1.0 + scale * rng.standard_normal(3) * dx
                v = scale * rng.standard_normal(2)
                got = O.limiter(u[0], u[1], u[2], v[0], v[1], dx, d)
                ref = brute_limiter(u[0], u[1], u[2], v[0], v[1], dx, d, 1e-6)
                vs = max(1.0, abs(ref["dq0"]), abs(ref["dq1"]), abs(ref["dq2"]))
                for k in ("dq0", "dq1", "dq2"):
                    assert abs(got[k] - ref[k]) < 1e-10 * vs, k
                bs = max(ref["beta0"], ref["beta1"], ref["beta2"], 1e-30)
                for k in ("beta0", "beta1", "beta2"):
                    assert abs(got[k] - ref[k]) <= 1e-10 * bs, (k, got[k], ref[k])
                for k in ("lambda0", "lambda1", "lambda2"):
                    assert abs(got[k] - ref[k]) < 1e-9
                assert abs(got["vt"] - ref["vt"]) < 1e-9 * vs


def test_limiter_exactness():
    """q_0'(x_i) is exact for quartic point data; the limited derivative is
    exact for linear data whatever the weights."""
    rng = np.random.default_rng(8)
    for _ in range(20):
        c = rng.standard_normal(5)
        dx = 10 ** rng.uniform(-2, 0)
        P = np.polynomial.Polynomial(c)
        dP = P.deriv()
        got = O.limiter(P(-dx), P(0.0), P(dx), dP(-dx), dP(dx), dx)
        assert abs(got["dq0"] - dP(0.0)) < 1e-11 * (1 + np.max(np.abs(c))) / dx
        a, b = rng.standard_normal(2)
        lin = O.limiter(a - b * dx, a, a + b * dx, b, b, dx, (0.3, 0.3, 0.4))
        assert abs(lin["vt"] - b) < 1e-12 * (1 + abs(b) + abs(a) / dx)
