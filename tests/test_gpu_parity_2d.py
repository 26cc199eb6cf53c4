"""GPU parity of the 2D path (x-sweep + y-sweep kernels through the C ABI)
against the oracle, and properties that hold at full size.

Tolerance scales as in the 1D tests, per direction: L^1 parts scale like
F/dx (F/dy), the derivative equations' own-direction parts like F/dx^2 and
the mixed parts like |eta|/dx, so each field's error is measured against
(F_x / dx^2 + F_y / dy^2) for L^2, L^3 and (F_x / dx + F_y / dy) for L^1;
limited derivatives against |U| / h. F is the size of the split fluxes.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2207_05258_gb300 import workloads as W
from _util import max_err, oracle_problem

pytestmark = pytest.mark.gpu
TOL = 1e-13


@pytest.fixture(scope="module")
def hw():
    from paper_2207_05258_gb300 import build
    build.build()
    from paper_2207_05258_gb300 import hweno
    return hweno


def dev(x, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to("cuda", dtype)


def flux_scale(w, U):
    """max over points of |f| + alpha |U| in x and y (numpy, for tolerances)."""
    U = U.reshape(w.m, -1)
    if w.equation == "burgers":
        a = np.max(np.abs(U))
        return 0.5 * a * a + a * a, 0.5 * a * a + a * a
    g = w.gas_gamma
    rho, m, n, E = U
    u, v = m / rho, n / rho
    p = (g - 1) * (E - 0.5 * (m * u + n * v))
    c = np.sqrt(g * p / rho)
    ax, ay = np.max(np.abs(u) + c), np.max(np.abs(v) + c)
    F = np.max(np.abs([m, m * u + p, m * v, (E + p) * u]))
    G = np.max(np.abs([n, n * u, n * v + p, (E + p) * v]))
    us = np.max(np.abs(U))
    return F + ax * us, G + ay * us


def rand_euler2d(nx, ny, seed, rough=True):
    rng = np.random.default_rng(seed)
    x = W.centers(0, 1, nx)[None, :]
    y = W.centers(0, 1, ny)[:, None]
    rho = 1 + 0.3 * np.sin(2 * np.pi * (x + 2 * y)) + (0.1 * rng.uniform(-1, 1, (ny, nx)) if rough else 0)
    u = 0.4 * np.cos(2 * np.pi * y) + (0.1 * rng.uniform(-1, 1, (ny, nx)) if rough else 0)
    v = -0.3 * np.sin(2 * np.pi * x) + (0.1 * rng.uniform(-1, 1, (ny, nx)) if rough else 0)
    p = 1 + 0.2 * np.cos(2 * np.pi * (x - y)) + (0.05 * rng.uniform(-1, 1, (ny, nx)) if rough else 0)
    U = W.euler_conserved(rho, u, p, 1.4, v=v)
    return U, rng.standard_normal(U.shape), rng.standard_normal(U.shape)


def make_w(equation, nx, ny, U, V, Wd, bc=("periodic",) * 4, inflow=(1.0, 0.3, -0.2, 2.6),
           x1=1.0, y1=1.0):
    return W.Workload("t2d", equation, 2, [nx], ny, 0.0, x1, 0.0, y1, 1.0, bc, U.ravel(),
                      V.ravel(), Wd.ravel(), inflow=inflow)


def check_rhs(hw, w, t=0.0, **opts):
    s = hw.Solver.from_workload(w, **opts)
    tt = torch.full((1,), t, dtype=torch.float64, device="cuda")
    r = s.rhs(dev(w.U), dev(w.V), dev(w.W), t=tt)
    torch.cuda.synchronize()
    s.sync_status()
    shp = (w.m, w.ny, w.nx[0])
    ref = O.rhs(oracle_problem(w, **opts), w.U, w.V, w.W, t=t)
    dx, dy = (w.x1 - w.x0) / w.nx[0], (w.y1 - w.y0) / w.ny
    Fx, Fy = flux_scale(w, w.U)
    us = np.max(np.abs(w.U))
    bounds = dict(L1=Fx / dx + Fy / dy, L2=Fx / dx ** 2 + Fy / dy ** 2,
                  L3=Fx / dx ** 2 + Fy / dy ** 2, Vt=us / dx, Wt=us / dy)
    for k, b in bounds.items():
        e = max_err(r[k].cpu().numpy().reshape(shp), ref[k])
        assert e <= TOL * b, (k, e, b)
    s.close()


@pytest.mark.parametrize("nx,ny", [(130, 23), (4, 4), (124, 7), (125, 8), (31, 50)])
def test_rhs_euler_periodic(hw, nx, ny):
    U, V, Wd = rand_euler2d(nx, ny, nx * 7 + ny)
    check_rhs(hw, make_w("euler", nx, ny, U, V, Wd))


@pytest.mark.parametrize("bc", [("outflow", "outflow", "reflective", "reflective"),
                                ("reflective", "inflow", "outflow", "inflow"),
                                ("inflow", "outflow", "periodic", "periodic")])
def test_rhs_euler_boundaries(hw, bc):
    U, V, Wd = rand_euler2d(130, 23, 3)
    check_rhs(hw, make_w("euler", 130, 23, U, V, Wd, bc=bc))


@pytest.mark.parametrize("opts", [dict(eig_avg=1), dict(limiter=0), dict(limiter=2),
                                  dict(lin_w=(0.5, 0.3, 0.2), lim_d=(0.6, 0.2, 0.2))])
def test_rhs_euler_options(hw, opts):
    U, V, Wd = rand_euler2d(60, 20, 4)
    check_rhs(hw, make_w("euler", 60, 20, U, V, Wd), **opts)


@pytest.mark.parametrize("bc", ["periodic", "reflective", "outflow"])
def test_rhs_burgers(hw, bc):
    rng = np.random.default_rng(5)
    nx, ny = 130, 23
    U = 0.3 + rng.uniform(-1, 1, (1, ny, nx))
    check_rhs(hw, make_w("burgers", nx, ny, U, rng.standard_normal(U.shape),
                         rng.standard_normal(U.shape), bc=(bc,) * 4, inflow=(0.5,)))


@pytest.mark.parametrize("t", [0.0, 0.013])
def test_rhs_double_mach_boundaries(hw, t):
    """DMR set-up with a non-zero V, W so that every ghost rule matters; at
    t > 0 the top boundary moves with the exact shock."""
    w = W.double_mach(130, 36)
    rng = np.random.default_rng(6)
    w.V = 0.1 * rng.standard_normal(w.U.shape)
    w.W = 0.1 * rng.standard_normal(w.U.shape)
    check_rhs(hw, w, t=t)


def gpu_run(hw, w, t_end, steps=None, precision="fp64", **opts):
    s = hw.Solver.from_workload(w, precision=precision, **opts)
    dt = torch.float64 if precision == "fp64" else torch.float32
    U, V, Wd = dev(w.U, dt), dev(w.V, dt), dev(w.W, dt)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    if steps is None:
        s.run(U, V, Wd, t, t_end)
    else:
        for _ in range(steps):
            s.step(U, V, Wd, t, t_end)
        s.sync_status()
    out = U.double().cpu().numpy(), V.double().cpu().numpy(), Wd.double().cpu().numpy(), float(t.item())
    s.close()
    return out


def compare(w, g, o, rtol_u, rtol_vw):
    shp = (w.m, w.ny, w.nx[0])
    eu = max_err(g[0].reshape(shp), o[0]) / np.max(np.abs(o[0]))
    ev = max_err(g[1].reshape(shp), o[1]) / max(np.max(np.abs(o[1])), 1e-300)
    ew = max_err(g[2].reshape(shp), o[2]) / max(np.max(np.abs(o[2])), 1e-300)
    assert eu <= rtol_u and ev <= rtol_vw and ew <= rtol_vw, (eu, ev, ew)
    assert abs(g[3] - o[3]) <= 1e-14 * max(o[3], 1e-300)
    return eu, ev, ew


@pytest.mark.parametrize("opts", [dict(), dict(dt_mode=1), dict(limiter=2, eig_avg=1)])
def test_one_step_euler(hw, opts):
    U, V, Wd = rand_euler2d(130, 23, 8)
    w = make_w("euler", 130, 23, U, V, Wd, bc=("outflow", "outflow", "reflective", "reflective"))
    g = gpu_run(hw, w, 1.0, steps=1, **opts)
    o = O.step(oracle_problem(w, **opts), w.U, w.V, w.W, 0.0, 1.0)
    compare(w, g, o[:3] + (o[3],), 1e-13, 1e-12)


def test_one_step_double_mach(hw):
    w = W.double_mach(130, 36)
    g = gpu_run(hw, w, 1.0, steps=2)
    P = oracle_problem(w)
    U, V, Wd, t, _ = O.run(P, w.U, w.V, w.W, 0.0, 1.0, max_steps=2)
    compare(w, g, (U, V, Wd, t), 1e-13, 1e-11)


def test_smooth_run_euler_config(hw):
    """2D Euler smooth periodic (rho = 1 + 0.2 sin(pi(x+y)), u = 0.7, v = 0.3)."""
    w = W.euler2d_smooth(32, t_end=0.2)
    g = gpu_run(hw, w, w.t_end)
    U, V, Wd, t, _ = O.run(oracle_problem(w), w.U, w.V, w.W, 0.0, w.t_end)
    compare(w, g, (U, V, Wd, t), 1e-10, 1e-10)


def test_smooth_run_burgers_example_3_8(hw):
    w = W.burgers2d_sine(40)
    g = gpu_run(hw, w, w.t_end)
    U, V, Wd, t, _ = O.run(oracle_problem(w), w.U, w.V, w.W, 0.0, w.t_end)
    compare(w, g, (U, V, Wd, t), 1e-10, 1e-10)


def test_shocked_run_burgers_example_3_10(hw):
    w = W.burgers2d_sine(40, t_end=1.5 / math.pi, dt_mode="cfl")
    g = gpu_run(hw, w, w.t_end)
    U, V, Wd, t, _ = O.run(oracle_problem(w), w.U, w.V, w.W, 0.0, w.t_end)
    compare(w, g, (U, V, Wd, t), 1e-8, 1e-8)


def test_shocked_run_double_mach_small(hw):
    w = W.double_mach(96, 24, t_end=0.02)
    g = gpu_run(hw, w, w.t_end)
    U, V, Wd, t, _ = O.run(oracle_problem(w), w.U, w.V, w.W, 0.0, w.t_end)
    compare(w, g, (U, V, Wd, t), 1e-8, 1e-8)


def test_full_size_double_mach_one_step(hw):
    """The 1920 x 480 double-Mach grid in the launch configuration of a full
    run, one step, against the oracle on the whole grid."""
    w = W.double_mach(1920, 480)
    g = gpu_run(hw, w, w.t_end, steps=1)
    U, V, Wd, t, _ = O.run(oracle_problem(w), w.U, w.V, w.W, 0.0, w.t_end, max_steps=1)
    compare(w, g, (U, V, Wd, t), 1e-13, 1e-11)


def test_full_size_periodic_translation_and_conservation(hw):
    """2048^2 periodic Euler: shifting the data by (dx, dy) = (3, 5) cells
    shifts the result bit for bit, and sum(U) is conserved."""
    n = 2048
    w = W.euler2d_smooth(n, dt_mode="cfl")
    g0 = gpu_run(hw, w, 1.0, steps=2)
    sh = lambda a: np.roll(np.roll(a.reshape(w.m, n, n), 5, axis=1), 3, axis=2)
    w2 = W.Workload(w.name, w.equation, 2, w.nx, w.ny, w.x0, w.x1, w.y0, w.y1, w.t_end, w.bc,
                    sh(w.U).ravel(), sh(w.V).ravel(), sh(w.W).ravel(), dt_mode="cfl")
    g1 = gpu_run(hw, w2, 1.0, steps=2)
    assert np.array_equal(g1[0].reshape(w.m, n, n), sh(g0[0]))
    assert np.array_equal(g1[1].reshape(w.m, n, n), sh(g0[1]))
    tot0 = w.U.reshape(w.m, -1).sum(axis=1)
    tot1 = g0[0].reshape(w.m, -1).sum(axis=1)
    assert np.all(np.abs(tot1 - tot0) <= 1e-12 * np.abs(w.U.reshape(w.m, -1)).sum(axis=1))


def test_2d_reduces_to_1d_on_gpu(hw):
    """y-independent data with v = 0 and W = 0: the 2D kernels give the 1D
    kernel's result (fixed dt: the 2D CFL step also counts the sound speed
    in y)."""
    n, ny = 200, 9
    w1 = W.riemann1d(n, (1.0, 0.1, 1.0), (0.3, -0.2, 0.4))
    U1, V1 = w1.instance(0)
    U2 = np.zeros((4, ny, n)); V2 = np.zeros((4, ny, n))
    for c2, c1 in ((0, 0), (1, 1), (3, 2)):
        U2[c2] = U1[c1][None, :]; V2[c2] = V1[c1][None, :]
    w2 = make_w("euler", n, ny, U2, V2, np.zeros_like(U2), bc=("outflow", "outflow", "periodic", "periodic"))
    g2 = gpu_run(hw, w2, 0.15, steps=5, dt_mode=2, dt_fixed=1e-3)
    s = hw.Solver.from_workload(w1, dt_mode=2, dt_fixed=1e-3)
    U, V = dev(w1.U), dev(w1.V)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(5):
        s.step(U, V, None, t, 0.15)
    g1 = U.cpu().numpy().reshape(3, n)
    G2 = g2[0].reshape(4, ny, n)
    for c2, c1 in ((0, 0), (1, 1), (3, 2)):
        assert np.max(np.abs(G2[c2] - g1[c1][None, :])) <= 1e-13 * np.max(np.abs(g1[c1]))
    assert np.max(np.abs(G2[2])) <= 1e-13


def test_fp32_error_2d(hw):
    """FP32 2D Euler smooth run: relative L-inf error against the FP64
    oracle, stated."""
    w = W.euler2d_smooth(32, t_end=0.2)
    g = gpu_run(hw, w, w.t_end, precision="fp32")
    U, _, _, _, _ = O.run(oracle_problem(w), w.U, w.V, w.W, 0.0, w.t_end)
    e = max_err(g[0].reshape(U.shape), U) / np.max(np.abs(U))
    print("fp32 2D Euler smooth 32^2 T=0.2: rel Linf(U) = %.3e" % e)
    assert e < 1e-4, e
