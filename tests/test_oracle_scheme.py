"""Scheme-level pins of the oracle: invariants and special cases that the
L-HWENO operators must satisfy whatever the implementation (Sec. 2).

* constant states give L = 0 exactly;
* periodic runs conserve sum(U) dx (the governing equation is in flux form,
  Eq. odeH); sum(V) is not conserved because the limiter replaces V;
* shifting a periodic grid shifts the result bit for bit;
* reflection symmetry x -> -x (Burgers with u -> -u; Euler with the normal
  momentum odd) maps the "+" fluxes onto the "-" fluxes, which pins the
  mirror procedure;
* 2D data that do not depend on y (or x) reduce the 2D scheme (Eq. ode2H with
  the mixed terms of Eq. mixed) to the 1D one;
* the operators reach their stated orders on smooth data: L^1 fifth order,
  the limited derivative fourth order (Sec. 2.2).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2207_05258_gb300 import workloads as W
from _util import oracle_problem

G = 1.4


def rand_euler1d(rng, n):
    x = W.centers(0, 2, n)
    rho = 1.0 + 0.3 * np.sin(np.pi * x + rng.uniform(0, 6)) + 0.05 * rng.standard_normal(n)
    u = 0.4 * np.cos(np.pi * x) + 0.05 * rng.standard_normal(n)
    p = 1.0 + 0.2 * np.sin(2 * np.pi * x) + 0.05 * rng.standard_normal(n)
    U = W.euler_conserved(rho, u, p, G)
    V = rng.standard_normal(U.shape)
    return U, V


def rand_euler2d(rng, nx, ny):
    rho = 1.0 + 0.2 * rng.uniform(-1, 1, (ny, nx))
    u, v = 0.4 * rng.uniform(-1, 1, (ny, nx)), 0.4 * rng.uniform(-1, 1, (ny, nx))
    p = 1.0 + 0.2 * rng.uniform(-1, 1, (ny, nx))
    U = W.euler_conserved(rho, u, p, G, v=v)
    return U, rng.standard_normal(U.shape), rng.standard_normal(U.shape)


def test_constant_state_is_steady():
    for P, shp in ((O.problem(O.EQ_BURGERS, 1, 16), (1, 16)),
                   (O.problem(O.EQ_EULER, 1, 16), (3, 16)),
                   (O.problem(O.EQ_EULER, 2, 12, 10), (4, 10, 12))):
        base = np.array([0.7] if shp[0] == 1 else ([1.3, 0.4, 2.5] if shp[0] == 3 else [1.3, 0.4, -0.2, 2.5]))
        U = np.broadcast_to(base.reshape((-1,) + (1,) * (len(shp) - 1)), shp).copy()
        Z = np.zeros(shp)
        r = O.rhs(P, U, Z, Z if P.dim == 2 else None)
        assert np.all(r["L1"] == 0.0) and np.all(r["L2"] == 0.0) and np.all(r["Vt"] == 0.0)
        if P.dim == 2:
            assert np.all(r["L3"] == 0.0) and np.all(r["Wt"] == 0.0)


@pytest.mark.parametrize("case", ["burgers1d", "euler1d", "euler2d", "burgers2d"])
def test_periodic_conservation(case):
    rng = np.random.default_rng(11)
    if case == "burgers1d":
        w = W.burgers1d_sine(64)
        P, U, V, Wd = oracle_problem(w), w.U, w.V, None
    elif case == "euler1d":
        P = O.problem(O.EQ_EULER, 1, 64, x0=0, x1=2)
        U, V = rand_euler1d(rng, 64)
        Wd = None
    elif case == "burgers2d":
        w = W.burgers2d_sine(16, dt_mode="cfl")
        P, U, V, Wd = oracle_problem(w), w.U, w.V, w.W
    else:
        P = O.problem(O.EQ_EULER, 2, 16, 12, x1=2, y1=2)
        U, V, Wd = rand_euler2d(rng, 16, 12)
    U = np.asarray(U).reshape((O.ncomp(P),) + ((P.ny, P.nx) if P.dim == 2 else (P.nx,)))
    tot0 = U.reshape(U.shape[0], -1).sum(axis=1)
    U1, V1, W1, t, k = O.run(P, U, V, Wd, 0.0, 1.0, max_steps=15)
    tot1 = U1.reshape(U1.shape[0], -1).sum(axis=1)
    scale = np.abs(U).reshape(U.shape[0], -1).sum(axis=1)
    assert k == 15
    assert np.all(np.abs(tot1 - tot0) <= 1e-13 * scale), (tot1 - tot0) / scale


def test_translation_equivariance_1d_and_2d():
    rng = np.random.default_rng(12)
    P = O.problem(O.EQ_EULER, 1, 40, x1=2)
    U, V = rand_euler1d(rng, 40)
    r0 = O.rhs(P, U, V)
    r1 = O.rhs(P, np.roll(U, 7, axis=1), np.roll(V, 7, axis=1))
    for k in ("L1", "L2", "Vt"):
        assert np.array_equal(r1[k], np.roll(r0[k], 7, axis=1))
    P2 = O.problem(O.EQ_EULER, 2, 12, 10, x1=2, y1=2)
    U, V, Wd = rand_euler2d(rng, 12, 10)
    r0 = O.rhs(P2, U, V, Wd)
    sh = lambda a: np.roll(np.roll(a, 3, axis=2), -4, axis=1)
    r1 = O.rhs(P2, sh(U), sh(V), sh(Wd))
    for k in ("L1", "L2", "L3", "Vt", "Wt"):
        assert np.array_equal(r1[k], sh(r0[k]))


def test_reflection_burgers_is_exact():
    """(x, u) -> (-x, -u) maps f^+ data onto mirrored f^- data exactly, so the
    reflected flux differences are bit-identical."""
    rng = np.random.default_rng(13)
    n = 48
    P = O.problem(O.EQ_BURGERS, 1, n, x1=2)
    U = rng.uniform(-1, 1.5, (1, n))
    V = 3 * rng.standard_normal((1, n))
    r0 = O.rhs(P, U, V)
    r1 = O.rhs(P, -U[:, ::-1].copy(), V[:, ::-1].copy())
    assert np.array_equal(r1["L1"], -r0["L1"][:, ::-1])
    assert np.array_equal(r1["L2"], r0["L2"][:, ::-1])
    # the limiter's sums associate differently after reflection: roundoff only
    assert np.max(np.abs(r1["Vt"] - r0["Vt"][:, ::-1])) < 1e-13 * np.max(np.abs(r0["Vt"]))


def test_reflection_euler1d():
    rng = np.random.default_rng(14)
    n = 48
    P = O.problem(O.EQ_EULER, 1, n, x1=2, bc=(O.BC_REFLECTIVE, O.BC_REFLECTIVE))
    S = np.array([1.0, -1.0, 1.0])[:, None]
    for bc in ((O.BC_PERIODIC, O.BC_PERIODIC), (O.BC_REFLECTIVE, O.BC_REFLECTIVE),
               (O.BC_OUTFLOW, O.BC_OUTFLOW)):
        P.bc[0], P.bc[1] = bc
        U, V = rand_euler1d(rng, n)
        r0 = O.rhs(P, U, V)
        r1 = O.rhs(P, (S * U)[:, ::-1].copy(), (-S * V)[:, ::-1].copy())
        sc = lambda a: np.max(np.abs(a))
        assert np.max(np.abs(r1["L1"] - (S * r0["L1"])[:, ::-1])) < 1e-12 * sc(r0["L1"])
        assert np.max(np.abs(r1["L2"] - (-S * r0["L2"])[:, ::-1])) < 1e-12 * sc(r0["L2"])
        assert np.max(np.abs(r1["Vt"] - (-S * r0["Vt"])[:, ::-1])) < 1e-12 * sc(r0["Vt"])


@pytest.mark.parametrize("axis", [0, 1])
def test_reflection_euler2d(axis):
    rng = np.random.default_rng(15 + axis)
    P = O.problem(O.EQ_EULER, 2, 14, 12, x1=2, y1=2)
    U, V, Wd = rand_euler2d(rng, 14, 12)
    S = np.array([1.0, -1.0, 1.0, 1.0] if axis == 0 else [1.0, 1.0, -1.0, 1.0])[:, None, None]
    flip = (lambda a: a[:, :, ::-1].copy()) if axis == 0 else (lambda a: a[:, ::-1, :].copy())
    sV, sW = (-1.0, 1.0) if axis == 0 else (1.0, -1.0)
    r0 = O.rhs(P, U, V, Wd)
    r1 = O.rhs(P, flip(S * U), flip(sV * S * V), flip(sW * S * Wd))
    for k, s in (("L1", 1.0), ("L2", sV), ("L3", sW), ("Vt", sV), ("Wt", sW)):
        ref = flip(s * S * r0[k])
        assert np.max(np.abs(r1[k] - ref)) < 1e-12 * np.max(np.abs(ref)), k


def test_2d_euler_reduces_to_1d():
    rng = np.random.default_rng(16)
    n, ny = 32, 6
    U1, V1 = rand_euler1d(rng, n)
    P1 = O.problem(O.EQ_EULER, 1, n, x1=2)
    r1 = O.rhs(P1, U1, V1)
    # y-independent data, v = 0, W = 0
    U2 = np.zeros((4, ny, n)); V2 = np.zeros((4, ny, n))
    for c2, c1 in ((0, 0), (1, 1), (3, 2)):
        U2[c2] = U1[c1][None, :]; V2[c2] = V1[c1][None, :]
    P2 = O.problem(O.EQ_EULER, 2, n, ny, x1=2, y1=1)
    r2 = O.rhs(P2, U2, V2, np.zeros_like(U2))
    for k in ("L1", "L2", "Vt"):
        sc = np.max(np.abs(r1[k]))
        for c2, c1 in ((0, 0), (1, 1), (3, 2)):
            assert np.max(np.abs(r2[k][c2] - r1[k][c1][None, :])) < 1e-13 * sc, k
        assert np.max(np.abs(r2[k][2])) < 1e-13 * sc
    assert np.max(np.abs(r2["L3"])) < 1e-13 and np.max(np.abs(r2["Wt"])) < 1e-13
    # x-independent data, u = 0, V = 0: the y-sweep against 1D
    U3 = np.zeros((4, n, ny)); W3 = np.zeros((4, n, ny))
    for c2, c1 in ((0, 0), (2, 1), (3, 2)):
        U3[c2] = U1[c1][:, None]; W3[c2] = V1[c1][:, None]
    P3 = O.problem(O.EQ_EULER, 2, ny, n, x1=1, y1=2)
    r3 = O.rhs(P3, U3, np.zeros_like(U3), W3)
    for k3, k1 in (("L1", "L1"), ("L3", "L2"), ("Wt", "Vt")):
        sc = np.max(np.abs(r1[k1]))
        for c2, c1 in ((0, 0), (2, 1), (3, 2)):
            assert np.max(np.abs(r3[k3][c2] - r1[k1][c1][:, None])) < 1e-13 * sc, k3


def test_2d_burgers_reduces_to_1d():
    n = 40
    w = W.burgers1d_sine(n)
    P1 = oracle_problem(w)
    r1 = O.rhs(P1, w.U, w.V)
    U2 = np.repeat(w.U.reshape(1, 1, n), 5, axis=1)
    V2 = np.repeat(w.V.reshape(1, 1, n), 5, axis=1)
    P2 = O.problem(O.EQ_BURGERS, 2, n, 5, x0=0, x1=2, y0=0, y1=1)
    r2 = O.rhs(P2, U2, V2, np.zeros_like(U2))
    for k in ("L1", "L2", "Vt"):
        assert np.max(np.abs(r2[k] - r1[k][:, None, :])) < 1e-13 * np.max(np.abs(r1[k]))
    assert np.all(r2["L3"] == 0.0) and np.all(r2["Wt"] == 0.0)


def test_rhs_and_limiter_orders():
    """L^1 = -f(u)_x + O(dx^5); the limited derivative = v + O(dx^4)."""
    e1, e2, e3 = [], [], []
    for n in (40, 80, 160):
        w = W.burgers1d_sine(n)
        r = O.rhs(oracle_problem(w), w.U, w.V)
        x = W.centers(0, 2, n)
        u, v, vx = 0.5 + np.sin(np.pi * x), np.pi * np.cos(np.pi * x), -np.pi ** 2 * np.sin(np.pi * x)
        e1.append(np.max(np.abs(r["L1"][0] + u * v)))
        e2.append(np.max(np.abs(r["L2"][0] + (v * v + u * vx))))
        e3.append(np.max(np.abs(r["Vt"][0] - v)))
    o1 = [math.log2(a / b) for a, b in zip(e1, e1[1:])]
    o2 = [math.log2(a / b) for a, b in zip(e2, e2[1:])]
    o3 = [math.log2(a / b) for a, b in zip(e3, e3[1:])]
    assert min(o1) > 4.7, o1
    assert min(o2) > 3.8, o2   # h-hat is O(dx^5) so its difference is O(dx^4)
    assert min(o3) > 3.7, o3


def test_limiter_off_keeps_derivative():
    rng = np.random.default_rng(17)
    P = O.problem(O.EQ_EULER, 1, 30, x1=2, limiter=0)
    U, V = rand_euler1d(rng, 30)
    assert np.array_equal(O.rhs(P, U, V)["Vt"], V)


def test_component_limiter_option():
    """limiter = 2 applies the scalar limiter to each component directly."""
    rng = np.random.default_rng(18)
    n = 20
    P = O.problem(O.EQ_EULER, 1, n, x1=2, limiter=2)
    U, V = rand_euler1d(rng, n)
    vt = O.rhs(P, U, V)["Vt"]
    dx = 2.0 / n
    for c in range(3):
        for i in (0, 5, n - 1):
            im, ip = (i - 1) % n, (i + 1) % n
            ref = O.limiter(U[c, im], U[c, i], U[c, ip], V[c, im], V[c, ip], dx)["vt"]
            assert vt[c, i] == ref


def test_run_lands_on_final_time():
    w = W.burgers1d_sine(50, t_end=0.1)
    U, V, _, t, k = O.run(oracle_problem(w), w.U, w.V, None, 0.0, w.t_end)
    assert t == w.t_end and k > 1
