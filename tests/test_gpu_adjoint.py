"""The discrete adjoint (hweno_adjoint_step and the checkpointed autograd
Function) against the oracle's forward-mode dual-number derivative: for a
seeded direction d and adjoint seed lam, <adjoint(lam), d> must equal
<lam, tangent(d)> with the same freezes (alpha per stage, dt of the run,
|.| branches of the forward state). Also against central finite differences
of the GPU forward (alpha not frozen there, so to a looser bound)."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2207_05258_gb300 import workloads as W
from _util import oracle_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hw():
    from paper_2207_05258_gb300 import build
    build.build()
    from paper_2207_05258_gb300 import hweno
    return hweno


def rough_batch(sizes, bc, seed):
    rng = np.random.default_rng(seed)
    Us, Vs = [], []
    for n in sizes:
        x = W.centers(0, 2, n)
        Us.append(0.4 + np.sin(np.pi * x + rng.uniform(0, 6)) + 0.1 * rng.standard_normal(n))
        Vs.append(np.pi * np.cos(np.pi * x) + rng.standard_normal(n))
    return W.Workload("rb", "burgers", 1, list(sizes), 1, 0.0, 2.0, 0.0, 1.0, 1.0,
                      (bc, bc, "periodic", "periodic"), np.concatenate(Us), np.concatenate(Vs),
                      inflow=(0.6, 0, 0, 0))


@pytest.mark.parametrize("bc", ["periodic", "outflow", "reflective", "inflow"])
def test_one_step_dot_product_against_dual_oracle(hw, bc):
    w = rough_batch([4, 31, 124, 125, 300], bc, 7)
    s = hw.Solver.from_workload(w)
    U, V = torch.from_numpy(w.U.copy()).cuda(), torch.from_numpy(w.V.copy()).cuda()
    t = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
    dt = torch.empty(w.batch, dtype=torch.float64, device="cuda")
    U1, V1 = U.clone(), V.clone()
    s.step(U1, V1, None, t, 1.0, dt)
    rng = np.random.default_rng(11)
    lamU = rng.standard_normal(w.U.size)
    lamV = rng.standard_normal(w.V.size)
    lU, lV = torch.from_numpy(lamU).cuda(), torch.from_numpy(lamV).cuda()
    s.adjoint_step(U, V, None, dt, lU, lV)
    s.sync_status()
    gU, gV = lU.cpu().numpy(), lV.cpu().numpy()
    off = 0
    for k, n in enumerate(w.nx):
        Uk, Vk = w.instance(k)
        dU, dV = rng.standard_normal(Uk.shape), rng.standard_normal(Vk.shape)
        out = O.run_tangent(oracle_problem(w, nx=n), Uk, Vk, None, dU, dV, None, 0.0, 1.0,
                            max_steps=1)
        lhs = float(np.dot(gU[off:off + n], dU.ravel()) + np.dot(gV[off:off + n], dV.ravel()))
        rhs = float(np.dot(lamU[off:off + n], out[3].ravel()) +
                    np.dot(lamV[off:off + n], out[4].ravel()))
        scale = np.sqrt(np.sum(lamU[off:off + n] ** 2 + lamV[off:off + n] ** 2) *
                        np.sum(out[3] ** 2 + out[4] ** 2)) + abs(rhs)
        assert abs(lhs - rhs) <= 1e-12 * scale, (k, n, lhs, rhs)
        off += n


def test_gradient_of_final_time_functional(hw):
    """J = sum_k sum_i u_k(T)^2 dx over a batch of smooth Burgers problems:
    the checkpointed adjoint gradient against the dual-number oracle along
    seeded directions, and against central differences of the GPU forward."""
    from paper_2207_05258_gb300.adjoint import run_to_time
    w = W.burgers_adjoint_batch(count=8, n=200)
    s = hw.Solver.from_workload(w)
    dx = 2.0 / 200
    U0 = torch.from_numpy(w.U.copy()).cuda().requires_grad_(True)
    V0 = torch.from_numpy(w.V.copy()).cuda().requires_grad_(True)
    UT, VT = run_to_time(U0, V0, s, w.t_end, 7)
    J = (UT * UT).sum() * dx
    J.backward()
    gU, gV = U0.grad.cpu().numpy(), V0.grad.cpu().numpy()
    rng = np.random.default_rng(21)
    for k in (0, 3, 7):
        Uk, Vk = w.instance(k)
        x = W.centers(0, 2, 200)
        dU = (0.1 * np.sin(3 * np.pi * x + rng.uniform(0, 6))).reshape(1, -1)
        dV = (0.3 * np.pi * np.cos(3 * np.pi * x)).reshape(1, -1)
        out = O.run_tangent(oracle_problem(w, nx=200), Uk, Vk, None, dU, dV, None, 0.0, w.t_end)
        dJ = float(np.sum(2.0 * out[0] * out[3]) * dx)
        adj = float(np.dot(gU[k * 200:(k + 1) * 200], dU.ravel()) +
                    np.dot(gV[k * 200:(k + 1) * 200], dV.ravel()))
        assert abs(adj - dJ) <= 1e-10 * abs(dJ), (k, adj, dJ)
        # central differences of the GPU forward (alpha recomputed there)
        eps = 1e-6
        Js = []
        for sgn in (1.0, -1.0):
            Ue, Ve = w.U.copy(), w.V.copy()
            Ue[k * 200:(k + 1) * 200] += sgn * eps * dU.ravel()
            Ve[k * 200:(k + 1) * 200] += sgn * eps * dV.ravel()
            Ut, Vt = torch.from_numpy(Ue).cuda(), torch.from_numpy(Ve).cuda()
            t = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
            s.run(Ut, Vt, None, t, w.t_end)
            Js.append(float((Ut[k * 200:(k + 1) * 200] ** 2).sum().item()) * dx)
        fd = (Js[0] - Js[1]) / (2 * eps)
        print("instance %d: adjoint %.12e dual %.12e fd %.12e" % (k, adj, dJ, fd))
        # the forward also responds through alpha = max|u| and dt, which the
        # adjoint freezes; on this smooth run that response stays below 1e-6 of
        # the Cauchy-Schwarz scale |grad J| |d| (the directions are nearly
        # orthogonal to the gradient, so dJ itself can be small)
        gk = np.concatenate([gU[k * 200:(k + 1) * 200], gV[k * 200:(k + 1) * 200]])
        scale = np.linalg.norm(gk) * np.linalg.norm(np.concatenate([dU.ravel(), dV.ravel()]))
        assert abs(adj - fd) <= 1e-5 * scale, (k, adj, fd, scale)


def test_checkpoint_interval_does_not_change_the_gradient(hw):
    from paper_2207_05258_gb300.adjoint import run_to_time
    w = W.burgers_adjoint_batch(count=3, n=128, t_end=0.05)
    grads = []
    for every in (1, 5, 1000):
        s = hw.Solver.from_workload(w)
        U0 = torch.from_numpy(w.U.copy()).cuda().requires_grad_(True)
        V0 = torch.from_numpy(w.V.copy()).cuda().requires_grad_(True)
        UT, VT = run_to_time(U0, V0, s, w.t_end, every)
        ((UT * UT).sum() + (VT * VT).sum() * 1e-3).backward()
        grads.append((U0.grad.clone(), V0.grad.clone()))
    for g in grads[1:]:
        assert torch.equal(g[0], grads[0][0]) and torch.equal(g[1], grads[0][1])


def euler_rough_batch(sizes, bc, seed, riemann_every=0):
    """Ragged batch of 1D Euler states on [0, 1]: smooth waves plus small
    seeded noise (positive density and pressure) and noisy derivatives; every
    `riemann_every`-th instance is a Riemann problem instead."""
    rng = np.random.default_rng(seed)
    Us, Vs = [], []
    for k, n in enumerate(sizes):
        x = W.centers(0, 1, n)
        if riemann_every and k % riemann_every == riemann_every - 1:
            lo = x < 0.5
            rho, u, p = (np.where(lo, 1.0, 0.125), np.where(lo, 0.2, -0.1),
                         np.where(lo, 1.0, 0.1))
            V = np.zeros((3, n))
        else:
            ph = rng.uniform(0, 6.3, 3)
            rho = 1 + 0.2 * np.sin(2 * np.pi * x + ph[0]) + 0.02 * rng.standard_normal(n)
            u = 0.3 * np.sin(2 * np.pi * x + ph[1]) + 0.02 * rng.standard_normal(n)
            p = 1 + 0.2 * np.cos(2 * np.pi * x + ph[2]) + 0.02 * rng.standard_normal(n)
            V = 0.5 * rng.standard_normal((3, n))
        Us.append(W.euler_conserved(rho, u, p, 1.4).ravel())
        Vs.append(V.ravel())
    return W.Workload("erb", "euler", 1, list(sizes), 1, 0.0, 1.0, 0.0, 1.0, 1.0,
                      (bc, bc, "periodic", "periodic"), np.concatenate(Us), np.concatenate(Vs),
                      inflow=(1.0, 0.2, 2.6, 0.0))


def _dot_check(hw, w, seed, tol, **opts):
    s = hw.Solver.from_workload(w, **opts)
    U, V = torch.from_numpy(w.U.copy()).cuda(), torch.from_numpy(w.V.copy()).cuda()
    t = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
    dt = torch.empty(w.batch, dtype=torch.float64, device="cuda")
    s.step(U.clone(), V.clone(), None, t, 1.0, dt)
    rng = np.random.default_rng(seed)
    lamU, lamV = rng.standard_normal(w.U.size), rng.standard_normal(w.V.size)
    lU, lV = torch.from_numpy(lamU).cuda(), torch.from_numpy(lamV).cuda()
    s.adjoint_step(U, V, None, dt, lU, lV)
    s.sync_status()
    gU, gV = lU.cpu().numpy(), lV.cpu().numpy()
    m, off = w.m, 0
    worst = 0.0
    for k, n in enumerate(w.nx):
        Uk, Vk = w.instance(k)
        dU, dV = rng.standard_normal(Uk.shape), rng.standard_normal(Vk.shape)
        out = O.run_tangent(oracle_problem(w, nx=n, **opts), Uk, Vk, None, dU, dV, None, 0.0,
                            1.0, max_steps=1)
        sl = slice(m * off, m * (off + n))
        lhs = float(np.dot(gU[sl], dU.ravel()) + np.dot(gV[sl], dV.ravel()))
        rhs = float(np.dot(lamU[sl], out[3].ravel()) + np.dot(lamV[sl], out[4].ravel()))
        scale = np.sqrt(np.sum(lamU[sl] ** 2 + lamV[sl] ** 2) *
                        np.sum(out[3] ** 2 + out[4] ** 2)) + abs(rhs)
        worst = max(worst, abs(lhs - rhs) / scale)
        assert abs(lhs - rhs) <= tol * scale, (k, n, lhs, rhs, scale)
        off += n
    return worst


@pytest.mark.parametrize("bc", ["periodic", "outflow", "reflective", "inflow"])
def test_euler_one_step_dot_product_against_dual_oracle(hw, bc):
    w = euler_rough_batch([4, 31, 124, 125, 300], bc, 3, riemann_every=3)
    worst = _dot_check(hw, w, 17, 1e-11)
    print("euler %s: worst relative dot-product mismatch %.2e" % (bc, worst))


@pytest.mark.parametrize("limiter", [0, 2])
def test_euler_limiter_options(hw, limiter):
    w = euler_rough_batch([50, 249], "outflow", 4, riemann_every=2)
    _dot_check(hw, w, 19, 1e-11, limiter=limiter)


def test_euler_gradient_through_checkpointed_run(hw):
    """J = sum rho(T)^2 dx over smooth periodic Euler problems: adjoint
    gradient against the dual-number oracle along seeded directions."""
    from paper_2207_05258_gb300.adjoint import run_to_time
    w = euler_rough_batch([96, 160], "periodic", 8)
    w.t_end = 0.05
    s = hw.Solver.from_workload(w)
    U0 = torch.from_numpy(w.U.copy()).cuda().requires_grad_(True)
    V0 = torch.from_numpy(w.V.copy()).cuda().requires_grad_(True)
    UT, VT = run_to_time(U0, V0, s, w.t_end, 4)
    off, J = 0, 0.0
    for n in w.nx:
        J = J + (UT[3 * off:3 * off + n] ** 2).sum() / n
        off += n
    J.backward()
    gU, gV = U0.grad.cpu().numpy(), V0.grad.cpu().numpy()
    rng = np.random.default_rng(23)
    off = 0
    for k, n in enumerate(w.nx):
        Uk, Vk = w.instance(k)
        dU, dV = 0.01 * rng.standard_normal(Uk.shape), 0.1 * rng.standard_normal(Vk.shape)
        out = O.run_tangent(oracle_problem(w, nx=n), Uk, Vk, None, dU, dV, None, 0.0, w.t_end)
        dJ = float(np.sum(2.0 * out[0][0] * out[3][0]) / n)
        sl = slice(3 * off, 3 * (off + n))
        adj = float(np.dot(gU[sl], dU.ravel()) + np.dot(gV[sl], dV.ravel()))
        scale = np.linalg.norm(np.concatenate([gU[sl], gV[sl]])) * np.linalg.norm(
            np.concatenate([dU.ravel(), dV.ravel()]))
        print("euler instance %d: adjoint %.12e dual %.12e" % (k, adj, dJ))
        assert abs(adj - dJ) <= 1e-10 * scale, (k, adj, dJ, scale)
        off += n


def test_burgers_without_limiter(hw):
    w = rough_batch([40, 130], "outflow", 9)
    s = hw.Solver.from_workload(w, limiter=0)
    U, V = torch.from_numpy(w.U.copy()).cuda(), torch.from_numpy(w.V.copy()).cuda()
    t = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
    dt = torch.empty(w.batch, dtype=torch.float64, device="cuda")
    s.step(U.clone(), V.clone(), None, t, 1.0, dt)
    rng = np.random.default_rng(5)
    lamU, lamV = rng.standard_normal(w.U.size), rng.standard_normal(w.V.size)
    lU, lV = torch.from_numpy(lamU).cuda(), torch.from_numpy(lamV).cuda()
    s.adjoint_step(U, V, None, dt, lU, lV)
    s.sync_status()
    gU, gV = lU.cpu().numpy(), lV.cpu().numpy()
    off = 0
    for k, n in enumerate(w.nx):
        Uk, Vk = w.instance(k)
        dU, dV = rng.standard_normal(Uk.shape), rng.standard_normal(Vk.shape)
        out = O.run_tangent(oracle_problem(w, nx=n, limiter=0), Uk, Vk, None, dU, dV, None,
                            0.0, 1.0, max_steps=1)
        lhs = float(np.dot(gU[off:off + n], dU.ravel()) + np.dot(gV[off:off + n], dV.ravel()))
        rhs = float(np.dot(lamU[off:off + n], out[3].ravel()) +
                    np.dot(lamV[off:off + n], out[4].ravel()))
        assert abs(lhs - rhs) <= 1e-12 * (abs(rhs) + np.sqrt(n)), (k, lhs, rhs)
        off += n


# ---------------------------------------------------------------------------
# 2D
# ---------------------------------------------------------------------------
def rough_2d(eq, nx, ny, bcx, bcy, seed):
    """2D state on [0,1]^2: smooth waves plus small seeded noise (Euler:
    positive density and pressure) and noisy derivatives V, W."""
    rng = np.random.default_rng(seed)
    x = W.centers(0, 1, nx)[None, :]
    y = W.centers(0, 1, ny)[:, None]
    ph = rng.uniform(0, 6.3, 4)
    noise = lambda: 0.02 * rng.standard_normal((ny, nx))
    if eq == "euler":
        rho = 1 + 0.2 * np.sin(2 * np.pi * (x + y) + ph[0]) + noise()
        u = 0.3 * np.sin(2 * np.pi * x + ph[1]) + noise()
        v = 0.2 * np.cos(2 * np.pi * y + ph[2]) + noise()
        p = 1 + 0.2 * np.cos(2 * np.pi * (x - y) + ph[3]) + noise()
        U = W.euler_conserved(rho, u, p, 1.4, v=v)
        m = 4
    else:
        U = (0.3 + np.sin(2 * np.pi * (x + y) + ph[0]) + 5 * noise())[None]
        m = 1
    V = 0.5 * rng.standard_normal((m, ny, nx))
    Wd = 0.5 * rng.standard_normal((m, ny, nx))
    return W.Workload("r2", eq, 2, [nx], ny, 0.0, 1.0, 0.0, 1.0, 1.0, (bcx, bcx, bcy, bcy),
                      U.ravel().copy(), V.ravel().copy(), Wd.ravel().copy(),
                      inflow=(1.0, 0.2, 0.1, 2.6) if eq == "euler" else (0.6, 0, 0, 0))


def _dot_check_2d(hw, w, seed, tol, pre_steps=0, **opts):
    s = hw.Solver.from_workload(w, **opts)
    U = torch.from_numpy(w.U.copy()).cuda()
    V = torch.from_numpy(w.V.copy()).cuda()
    Wd = torch.from_numpy(w.W.copy()).cuda()
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(pre_steps):
        s.step(U, V, Wd, t, 1.0)
    t0 = t.clone()
    dt = torch.empty(1, dtype=torch.float64, device="cuda")
    s.step(U.clone(), V.clone(), Wd.clone(), t.clone(), 1.0, dt)
    rng = np.random.default_rng(seed)
    lam = [rng.standard_normal(w.U.size) for _ in range(3)]
    lt = [torch.from_numpy(x).cuda() for x in lam]
    s.adjoint_step(U, V, Wd, dt, lt[0], lt[1], lt[2], t=t0)
    s.sync_status()
    g = [x.cpu().numpy() for x in lt]
    d = [rng.standard_normal(w.U.size) for _ in range(3)]
    oopts = dict(opts)
    if "adj_frozen_weights" in oopts:  # the oracle's name for the same reading
        oopts["freeze_weights"] = oopts.pop("adj_frozen_weights")
    out = O.run_tangent(oracle_problem(w, **oopts), U.cpu().numpy(), V.cpu().numpy(),
                        Wd.cpu().numpy(), d[0], d[1], d[2], float(t0.item()), 1.0, max_steps=1)
    lhs = sum(float(np.dot(g[i], d[i])) for i in range(3))
    tan = [out[3].ravel(), out[4].ravel(), out[5].ravel()]
    rhs = sum(float(np.dot(lam[i], tan[i])) for i in range(3))
    scale = np.sqrt(sum(np.sum(x ** 2) for x in lam) * sum(np.sum(x ** 2) for x in tan)) + abs(rhs)
    assert abs(lhs - rhs) <= tol * scale, (lhs, rhs, scale)
    return abs(lhs - rhs) / scale


@pytest.mark.parametrize("case", [
    ("euler", 130, 128, "periodic", "periodic"),
    ("euler", 40, 130, "reflective", "outflow"),
    ("euler", 36, 28, "inflow", "reflective"),
    ("burgers", 130, 20, "periodic", "periodic"),
    ("burgers", 30, 40, "reflective", "outflow"),
])
def test_2d_one_step_dot_product_against_dual_oracle(hw, case):
    eq, nx, ny, bcx, bcy = case
    w = rough_2d(eq, nx, ny, bcx, bcy, 31)
    r = _dot_check_2d(hw, w, 41, 1e-11)
    print("2D %s %dx%d %s/%s: relative mismatch %.2e" % (eq, nx, ny, bcx, bcy, r))


@pytest.mark.parametrize("limiter", [0, 2])
def test_2d_euler_limiter_options(hw, limiter):
    w = rough_2d("euler", 30, 26, "outflow", "periodic", 32)
    _dot_check_2d(hw, w, 43, 1e-11, limiter=limiter)


def test_2d_double_mach_boundaries_at_positive_time(hw):
    """Double-Mach set-up (inflow left, outflow right, reflecting wall from
    x = 1/6 on the bottom, exact moving shock on the top) a few steps in, so
    that the top boundary's stage times matter."""
    w = W.double_mach(64, 16)
    r = _dot_check_2d(hw, w, 47, 1e-10, pre_steps=3)
    print("double Mach 64x16: relative mismatch %.2e" % r)


def test_2d_gradient_through_checkpointed_run(hw):
    from paper_2207_05258_gb300.adjoint import run_to_time
    w = rough_2d("euler", 24, 20, "periodic", "periodic", 33)
    t_end = 0.02
    s = hw.Solver.from_workload(w)
    U0 = torch.from_numpy(w.U.copy()).cuda().requires_grad_(True)
    V0 = torch.from_numpy(w.V.copy()).cuda().requires_grad_(True)
    W0 = torch.from_numpy(w.W.copy()).cuda().requires_grad_(True)
    UT, VT, WT = run_to_time(U0, V0, s, t_end, 3, W0=W0)
    n = 24 * 20
    J = (UT[:n] ** 2).sum() / n + 1e-3 * (VT * WT).sum()
    J.backward()
    g = [x.grad.cpu().numpy() for x in (U0, V0, W0)]
    rng = np.random.default_rng(51)
    d = [0.01 * rng.standard_normal(w.U.size) for _ in range(3)]
    out = O.run_tangent(oracle_problem(w), w.U, w.V, w.W, d[0], d[1], d[2], 0.0, t_end)
    UTo, VTo, WTo = (x.ravel() for x in out[:3])
    dU, dV, dW = (x.ravel() for x in out[3:6])
    dJ = float(np.sum(2 * UTo[:n] * dU[:n]) / n + 1e-3 * np.sum(dV * WTo + VTo * dW))
    adj = sum(float(np.dot(g[i], d[i])) for i in range(3))
    scale = np.sqrt(sum(np.sum(x ** 2) for x in g) * sum(np.sum(x ** 2) for x in d))
    print("2D gradient: adjoint %.12e dual %.12e" % (adj, dJ))
    assert abs(adj - dJ) <= 1e-10 * scale, (adj, dJ, scale)


# ---------------------------------------------------------------------------
# frozen-weights mode (adj_frozen_weights = 1) against the oracle's tangent
# with the weights held (freeze_weights = 1)
# ---------------------------------------------------------------------------
def test_frozen_weights_1d_burgers_and_euler(hw):
    for w in (rough_batch([31, 124, 300], "outflow", 61),
              euler_rough_batch([31, 125, 300], "reflective", 62, riemann_every=2)):
        s = hw.Solver.from_workload(w, adj_frozen_weights=1)
        U, V = torch.from_numpy(w.U.copy()).cuda(), torch.from_numpy(w.V.copy()).cuda()
        t = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
        dt = torch.empty(w.batch, dtype=torch.float64, device="cuda")
        s.step(U.clone(), V.clone(), None, t, 1.0, dt)
        rng = np.random.default_rng(63)
        lamU, lamV = rng.standard_normal(w.U.size), rng.standard_normal(w.V.size)
        lU, lV = torch.from_numpy(lamU).cuda(), torch.from_numpy(lamV).cuda()
        s.adjoint_step(U, V, None, dt, lU, lV)
        s.sync_status()
        gU, gV = lU.cpu().numpy(), lV.cpu().numpy()
        m, off = w.m, 0
        for k, n in enumerate(w.nx):
            Uk, Vk = w.instance(k)
            dU, dV = rng.standard_normal(Uk.shape), rng.standard_normal(Vk.shape)
            out = O.run_tangent(oracle_problem(w, nx=n, freeze_weights=1), Uk, Vk, None, dU, dV,
                                None, 0.0, 1.0, max_steps=1)
            full = O.run_tangent(oracle_problem(w, nx=n), Uk, Vk, None, dU, dV, None, 0.0, 1.0,
                                 max_steps=1)
            sl = slice(m * off, m * (off + n))
            lhs = float(np.dot(gU[sl], dU.ravel()) + np.dot(gV[sl], dV.ravel()))
            rhs = float(np.dot(lamU[sl], out[3].ravel()) + np.dot(lamV[sl], out[4].ravel()))
            rfull = float(np.dot(lamU[sl], full[3].ravel()) + np.dot(lamV[sl], full[4].ravel()))
            scale = np.sqrt(np.sum(lamU[sl] ** 2 + lamV[sl] ** 2) *
                            np.sum(out[3] ** 2 + out[4] ** 2)) + abs(rhs)
            assert abs(lhs - rhs) <= 1e-11 * scale, (w.equation, k, lhs, rhs)
            if w.equation == "euler" and k == 1:  # a Riemann instance: freezing matters
                assert abs(rfull - rhs) > 1e-6 * scale
            off += n


def test_frozen_weights_2d_euler(hw):
    w = rough_2d("euler", 40, 30, "periodic", "outflow", 64)
    r = _dot_check_2d(hw, w, 65, 1e-11, adj_frozen_weights=1)
    print("2D frozen weights: relative mismatch %.2e" % r)


# ---------------------------------------------------------------------------
# step records (hweno_step_record / hweno_adjoint_step_recorded): the adjoint
# without its replay gives the bits of the replaying adjoint
# ---------------------------------------------------------------------------
def _recorded_vs_replayed(hw, w, steps, t_end, two):
    s = hw.Solver.from_workload(w)
    dev = lambda x: torch.from_numpy(x.copy()).cuda()
    U, V = dev(w.U), dev(w.V)
    Wd = dev(w.W) if two else None
    t = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
    for _ in range(steps):  # move away from the initial data
        s.step(U, V, Wd, t, t_end)
    U0, V0 = U.clone(), V.clone()
    W0 = Wd.clone() if two else None
    t0 = t.clone()
    dt = torch.empty(w.batch, dtype=torch.float64, device="cuda")
    rec = s.new_record()
    s.step_record(U, V, Wd, t, t_end, rec, dt)
    rng = np.random.default_rng(5)
    lam = [torch.from_numpy(rng.standard_normal(w.U.size)).cuda() for _ in range(3 if two else 2)]
    a = [x.clone() for x in lam]
    b = [x.clone() for x in lam]
    s.adjoint_step(U0, V0, W0, dt, *a[:2], a[2] if two else None, t=t0)
    assert s.launches_last_call == (11 if two else 6)
    s.adjoint_step(U0, V0, W0, dt, *b[:2], b[2] if two else None, t=t0, record=rec)
    assert s.launches_last_call == (6 if two else 3)
    s.sync_status()
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    s.close()


def test_recorded_adjoint_1d_burgers(hw):
    w = rough_batch([40, 123, 124, 125, 300], "periodic", 61)
    _recorded_vs_replayed(hw, w, 2, 0.05, False)


def test_recorded_adjoint_1d_euler_with_finished_instances(hw):
    w = euler_rough_batch([40, 200, 130], "outflow", 62)
    _recorded_vs_replayed(hw, w, 3, 0.01, False)  # the 40-point instance lands on t_end early


@pytest.mark.parametrize("case", [("euler", 130, 128, "periodic", "periodic"),
                                  ("euler", 40, 36, "reflective", "outflow"),
                                  ("burgers", 30, 40, "periodic", "periodic")])
def test_recorded_adjoint_2d(hw, case):
    eq, nx, ny, bcx, bcy = case
    w = rough_2d(eq, nx, ny, bcx, bcy, 63)
    _recorded_vs_replayed(hw, w, 2, 1.0, True)


def test_record_arguments(hw):
    w = rough_batch([64], "periodic", 64)
    s = hw.Solver.from_workload(w)
    assert s.record_bytes >= 4 * 64 * 8 and s.record_bytes % 256 == 0
    U = torch.from_numpy(w.U.copy()).cuda()
    V = torch.from_numpy(w.V.copy()).cuda()
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(hw.HwenoError) as e:
        s.step_record(U, V, None, t, 1.0, None)
    assert e.value.code == hw.EINVAL
    s.close()
    f = hw.Solver.from_workload(w, precision="fp32")
    rec = torch.empty(4096, dtype=torch.uint8, device="cuda")
    with pytest.raises(hw.HwenoError) as e:
        f.step_record(U.float(), V.float(), None, t, 1.0, rec)
    assert e.value.code == hw.ENOTSUP
    f.close()


def test_recorded_adjoint_after_a_cluster_step(hw):
    """A record taken by the cluster step (fused_small = 2) holds the stage
    states that step computed; its adjoint matches the replaying adjoint
    (which recomputes them with the tiled kernels) to rounding."""
    w = rough_batch([40, 123, 300], "periodic", 65)
    s = hw.Solver.from_workload(w, fused_small=2)
    U = torch.from_numpy(w.U.copy()).cuda()
    V = torch.from_numpy(w.V.copy()).cuda()
    t = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
    U0, V0, t0 = U.clone(), V.clone(), t.clone()
    dt = torch.empty(w.batch, dtype=torch.float64, device="cuda")
    rec = s.new_record()
    s.step_record(U, V, None, t, 0.05, rec, dt)
    rng = np.random.default_rng(6)
    lam = [torch.from_numpy(rng.standard_normal(w.U.size)).cuda() for _ in range(2)]
    a = [x.clone() for x in lam]
    b = [x.clone() for x in lam]
    s.adjoint_step(U0, V0, None, dt, a[0], a[1], t=t0)
    s.adjoint_step(U0, V0, None, dt, b[0], b[1], t=t0, record=rec)
    s.sync_status()
    for x, y in zip(a, b):
        assert float((x - y).abs().max()) <= 1e-12 * float(x.abs().max())
    s.close()
