"""Exact solutions used to pin the oracle (TEST INFRASTRUCTURE).

* Burgers: u(x, t) = u0(x - u t) solved by Newton's method (smooth for t
  below the breaking time 1/max(-u0')), the classical method of
  characteristics.
* Euler, smooth translation: density advected at the constant velocity with
  constant pressure (Examples 3.2 and 3.9 of the paper).
* Euler, Riemann problem: the exact solver of Toro ("Riemann Solvers and
  Numerical Methods for Fluid Dynamics", Ch. 4): Newton iteration on the
  pressure function for p*, then sampling of the self-similar solution.
* Oblique-shock state: the Rankine-Hugoniot relations for a normal shock of
  Mach number M moving into gas at rest.
"""
from __future__ import annotations

import numpy as np


def burgers_characteristics(x, t, u0, du0, speed=1.0, iters=60):
    """Solve u = u0(x - speed*u*t) pointwise by Newton's method."""
    x = np.asarray(x, dtype=np.float64)
    u = u0(x)
    for _ in range(iters):
        xi = x - speed * u * t
        F = u - u0(xi)
        dF = 1.0 + du0(xi) * speed * t
        du = F / dF
        u = u - du
        if np.max(np.abs(du)) < 1e-15:
            break
    return u


def riemann_exact(left, right, gamma, x, t, x0=0.5):
    """Exact solution (rho, u, p) of the 1D Euler Riemann problem at (x, t).

    left, right: primitive states (rho, u, p)."""
    rl, ul, pl = map(float, left)
    rr, ur, pr = map(float, right)
    g = float(gamma)
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    if 2.0 / (g - 1.0) * (cl + cr) <= ur - ul:
        raise ValueError("vacuum is generated")

    def fk(p, rk, pk, ck):
        if p > pk:  # shock
            A, B = 2.0 / ((g + 1.0) * rk), (g - 1.0) / (g + 1.0) * pk
            s = np.sqrt(A / (p + B))
            return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (B + p))
        pr_ = p / pk  # rarefaction
        f = 2.0 * ck / (g - 1.0) * (pr_ ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rk * ck) * pr_ ** (-(g + 1.0) / (2.0 * g))
        return f, df

    # initial guess: linearised (primitive-variable) solver, floored
    p = max(1e-8, 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr))
    for _ in range(100):
        f1, d1 = fk(p, rl, pl, cl)
        f2, d2 = fk(p, rr, pr, cr)
        pn = p - (f1 + f2 + ur - ul) / (d1 + d2)
        pn = max(pn, 1e-10)
        if abs(pn - p) / (0.5 * (pn + p)) < 1e-15:
            p = pn
            break
        p = pn
    ps = p
    us = 0.5 * (ul + ur) + 0.5 * (fk(ps, rr, pr, cr)[0] - fk(ps, rl, pl, cl)[0])

    x = np.asarray(x, dtype=np.float64)
    rho, u, pp = np.empty_like(x), np.empty_like(x), np.empty_like(x)
    gm1, gp1 = g - 1.0, g + 1.0
    for k, xx in enumerate(x):
        S = (xx - x0) / t if t > 0 else (-np.inf if xx < x0 else np.inf)
        if S <= us:  # left of contact
            if ps > pl:  # left shock
                SL = ul - cl * np.sqrt(gp1 / (2 * g) * ps / pl + gm1 / (2 * g))
                if S <= SL:
                    st = (rl, ul, pl)
                else:
                    r = rl * (ps / pl + gm1 / gp1) / (gm1 / gp1 * ps / pl + 1.0)
                    st = (r, us, ps)
            else:  # left rarefaction
                SHL = ul - cl
                csl = cl * (ps / pl) ** (gm1 / (2 * g))
                STL = us - csl
                if S <= SHL:
                    st = (rl, ul, pl)
                elif S >= STL:
                    st = (rl * (ps / pl) ** (1.0 / g), us, ps)
                else:
                    c = 2.0 / gp1 * (cl + gm1 / 2.0 * (ul - S))
                    uu = 2.0 / gp1 * (cl + gm1 / 2.0 * ul + S)
                    r = rl * (c / cl) ** (2.0 / gm1)
                    st = (r, uu, pl * (c / cl) ** (2.0 * g / gm1))
        else:  # right of contact
            if ps > pr:  # right shock
                SR = ur + cr * np.sqrt(gp1 / (2 * g) * ps / pr + gm1 / (2 * g))
                if S >= SR:
                    st = (rr, ur, pr)
                else:
                    r = rr * (ps / pr + gm1 / gp1) / (gm1 / gp1 * ps / pr + 1.0)
                    st = (r, us, ps)
            else:  # right rarefaction
                SHR = ur + cr
                csr = cr * (ps / pr) ** (gm1 / (2 * g))
                STR = us + csr
                if S >= SHR:
                    st = (rr, ur, pr)
                elif S <= STR:
                    st = (rr * (ps / pr) ** (1.0 / g), us, ps)
                else:
                    c = 2.0 / gp1 * (cr - gm1 / 2.0 * (ur - S))
                    uu = 2.0 / gp1 * (-cr + gm1 / 2.0 * ur + S)
                    r = rr * (c / cr) ** (2.0 / gm1)
                    st = (r, uu, pr * (c / cr) ** (2.0 * g / gm1))
        rho[k], u[k], pp[k] = st
    return rho, u, pp, ps, us


def normal_shock_post_state(mach, rho1, p1, gamma):
    """Post-shock (rho2, p2, |u2|) behind a normal shock of Mach number `mach`
    moving into gas (rho1, p1) at rest (Rankine-Hugoniot)."""
    g, M = float(gamma), float(mach)
    c1 = np.sqrt(g * p1 / rho1)
    rho2 = rho1 * (g + 1.0) * M * M / ((g - 1.0) * M * M + 2.0)
    p2 = p1 * (2.0 * g * M * M - (g - 1.0)) / (g + 1.0)
    u2 = M * c1 * (1.0 - rho1 / rho2)  # lab-frame speed of the shocked gas
    return rho2, p2, u2


# ---------------------------------------------------------------------------
# Buckley-Leverett (Example 3.4): f(u) = 4u^2 / (4u^2 + (1 - u)^2), on
# [-1, 1] with u0 = 1 on [-1/2, 0], 0 elsewhere.
#
# Each jump is a Riemann problem whose entropy solution follows the convex
# hull of f between the two states (Oleinik): for the fall 1 -> 0 at x = 0,
# the upper concave envelope of f on [0, 1] is f on [u_a, 1] and the tangent
# from (0, 0), touching f where f'(u) u = f(u); with D = 5u^2 - 2u + 1 that
# is 2(1 - u) = D, i.e. u_a = 1/sqrt(5): a rarefaction (x/t = f'(u), u from 1
# down to u_a) followed by a shock to 0 at speed f(u_a)/u_a. For the rise
# 0 -> 1 at x = -1/2 the lower convex envelope is f on [0, u_b] and the
# tangent to (1, 1), touching where f'(u)(1 - u) = 1 - f(u), i.e. 8u = D,
# u_b = 1 - 2/sqrt(5): a rarefaction (x/t = f'(u), u from 0 up to u_b) then a
# shock to 1 at speed f'(u_b). The two waves are independent while the left
# shock has not reached the right fan's tail at x = 0 (f'(1) = 0), i.e. for
# t < 1/2 / f'(u_b) ~ 0.472, which covers T = 0.4.
# ---------------------------------------------------------------------------
def bl_f(u):
    return 4.0 * u * u / (4.0 * u * u + (1.0 - u) ** 2)


def bl_df(u):
    D = 4.0 * u * u + (1.0 - u) ** 2
    return 8.0 * u * (1.0 - u) / (D * D)


def _bl_invert(xi, lo, hi, iters=200):
    """u in [lo, hi] with f'(u) = xi, f' monotone on [lo, hi] (bisection)."""
    a, b = lo, hi
    fa = bl_df(a) - xi
    for _ in range(iters):
        m = 0.5 * (a + b)
        fm = bl_df(m) - xi
        if (fm > 0) == (fa > 0):
            a, fa = m, fm
        else:
            b = m
    return 0.5 * (a + b)


def buckley_leverett_exact(x, t):
    """Entropy solution of Example 3.4 at time t < 0.47 on points x."""
    x = np.asarray(x, dtype=np.float64)
    u_a = 1.0 / np.sqrt(5.0)
    u_b = 1.0 - 2.0 / np.sqrt(5.0)
    s_a = bl_f(u_a) / u_a          # shock speed of the fall at x = 0
    s_b = bl_df(u_b)               # shock speed of the rise at x = -1/2
    assert t * s_b < 0.5, "the waves interact after t = 0.5 / f'(u_b)"
    u = np.zeros_like(x)
    for k, xk in enumerate(x):
        if xk < -0.5:
            u[k] = 0.0
        elif xk < -0.5 + s_b * t:   # rise: fan u in [0, u_b], f' increasing there
            u[k] = _bl_invert((xk + 0.5) / t, 0.0, u_b) if t > 0 else 0.0
        elif xk < 0.0:
            u[k] = 1.0
        elif xk < s_a * t:          # fall: fan u in [u_a, 1], f' decreasing there
            u[k] = _bl_invert(xk / t, u_a, 1.0)
        else:
            u[k] = 0.0
    return u
