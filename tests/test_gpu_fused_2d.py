"""GPU parity of the fused 2D stage kernel (one launch per stage computing the
x and y parts of a 16 x 7 block of points, option fused_2d = 1) against the
oracle and against the split form (x-sweep then y-sweep), through the C ABI.

The fused kernel evaluates the same x and y interface fluxes and point terms
as the two sweeps, in the same order per point, so both forms agree with the
oracle to the 2D parity tolerances (one step: 1e-13 relative in U, 1e-11 in
V and W). Grids are ragged against the 16 x 7 block (130 x 23, 31 x 50,
4 x 4, 124 x 7, 125 x 8) and every boundary kind is covered, double Mach
included.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2207_05258_gb300 import workloads as W
from _util import max_err, oracle_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hw():
    from paper_2207_05258_gb300 import build
    build.build()
    from paper_2207_05258_gb300 import hweno
    return hweno


def dev(x, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to("cuda", dtype)


def rand_2d(eq, nx, ny, seed):
    rng = np.random.default_rng(seed)
    x = W.centers(0, 1, nx)[None, :]
    y = W.centers(0, 1, ny)[:, None]
    n = lambda a: a * rng.uniform(-1, 1, (ny, nx))
    if eq == "euler":
        rho = 1 + 0.3 * np.sin(2 * np.pi * (x + 2 * y)) + n(0.1)
        u = 0.4 * np.cos(2 * np.pi * y) + n(0.1)
        v = -0.3 * np.sin(2 * np.pi * x) + n(0.1)
        p = 1 + 0.2 * np.cos(2 * np.pi * (x - y)) + n(0.05)
        U = W.euler_conserved(rho, u, p, 1.4, v=v)
    else:
        U = (0.3 + np.sin(2 * np.pi * (x + y)) + n(0.2))[None]
    return U, rng.standard_normal(U.shape), rng.standard_normal(U.shape)


def make_w(eq, nx, ny, bc, seed):
    U, V, Wd = rand_2d(eq, nx, ny, seed)
    inflow = (1.0, 0.3, -0.2, 2.6) if eq == "euler" else (0.7, 0, 0, 0)
    return W.Workload("f2d", eq, 2, [nx], ny, 0.0, 1.0, 0.0, 1.0, 1.0, bc, U.ravel(),
                      V.ravel(), Wd.ravel(), inflow=inflow)


def gpu_steps(hw, w, steps, t_end, precision="fp64", **opts):
    s = hw.Solver.from_workload(w, precision=precision, **opts)
    dt = torch.float64 if precision == "fp64" else torch.float32
    U, V, Wd = dev(w.U, dt), dev(w.V, dt), dev(w.W, dt)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    launches = []
    if steps is None:
        s.run(U, V, Wd, t, t_end)
    else:
        for _ in range(steps):
            s.step(U, V, Wd, t, t_end)
            launches.append(s.launches_last_call)
    s.sync_status()
    out = (U.double().cpu().numpy(), V.double().cpu().numpy(), Wd.double().cpu().numpy(),
           float(t.item()))
    s.close()
    return out, launches


def rel(g, o, shp):
    return max_err(g.reshape(shp), o) / max(np.max(np.abs(o)), 1e-300)


def check(w, g, o, rtol_u, rtol_vw):
    shp = (w.m, w.ny, w.nx[0])
    eu, ev, ew = rel(g[0], o[0], shp), rel(g[1], o[1], shp), rel(g[2], o[2], shp)
    assert eu <= rtol_u and ev <= rtol_vw and ew <= rtol_vw, (eu, ev, ew)
    assert abs(g[3] - o[3]) <= 1e-14 * max(o[3], 1e-300)


GRIDS = [(130, 23), (31, 50), (4, 4), (124, 7), (125, 8)]
BCS = [("periodic",) * 4,
       ("outflow", "outflow", "reflective", "reflective"),
       ("reflective", "reflective", "outflow", "outflow"),
       ("inflow", "outflow", "periodic", "periodic")]


@pytest.mark.parametrize("nx,ny", GRIDS)
@pytest.mark.parametrize("eq", ["euler", "burgers"])
def test_fused_two_steps_vs_oracle_periodic(hw, eq, nx, ny):
    w = make_w(eq, nx, ny, BCS[0], 11 + nx)
    g, launches = gpu_steps(hw, w, 2, 1.0, fused_2d=1)
    assert launches == [5, 5]
    U, V, Wd, t, _ = O.run(oracle_problem(w), w.U, w.V, w.W, 0.0, 1.0, max_steps=2)
    check(w, g, (U, V, Wd, t), 1e-13, 1e-11)


@pytest.mark.parametrize("bc", BCS[1:])
@pytest.mark.parametrize("eq", ["euler", "burgers"])
def test_fused_boundaries_vs_oracle(hw, eq, bc):
    w = make_w(eq, 130, 23, bc, 5)
    g, _ = gpu_steps(hw, w, 2, 1.0, fused_2d=1)
    U, V, Wd, t, _ = O.run(oracle_problem(w), w.U, w.V, w.W, 0.0, 1.0, max_steps=2)
    check(w, g, (U, V, Wd, t), 1e-13, 1e-11)


@pytest.mark.parametrize("opts", [dict(dt_mode=1), dict(limiter=2, eig_avg=1), dict(limiter=0)])
def test_fused_options_vs_oracle(hw, opts):
    w = make_w("euler", 31, 50, BCS[1], 9)
    g, _ = gpu_steps(hw, w, 1, 1.0, fused_2d=1, **opts)
    o = O.step(oracle_problem(w, **opts), w.U, w.V, w.W, 0.0, 1.0)
    check(w, g, o[:4], 1e-13, 1e-11)


def test_fused_double_mach_vs_oracle(hw):
    """The double Mach boundaries (time-dependent top wall, reflective wedge)."""
    w = W.double_mach(130, 36)
    g, _ = gpu_steps(hw, w, 2, 1.0, fused_2d=1)
    U, V, Wd, t, _ = O.run(oracle_problem(w), w.U, w.V, w.W, 0.0, 1.0, max_steps=2)
    check(w, g, (U, V, Wd, t), 1e-13, 1e-11)


@pytest.mark.parametrize("nx,ny", GRIDS)
def test_fused_matches_split(hw, nx, ny):
    """Fused and split forms: the same result up to rounding, over five steps
    with the wall boundaries."""
    w = make_w("euler", nx, ny, BCS[1], 3 + ny)
    a, la = gpu_steps(hw, w, 5, 1.0, fused_2d=0)
    b, lb = gpu_steps(hw, w, 5, 1.0, fused_2d=1)
    assert la == [8] * 5 and lb == [5] * 5
    shp = (w.m, ny, nx)
    for x, y in zip(a[:3], b[:3]):
        assert rel(y, x.reshape(shp), shp) <= 1e-12
    assert abs(a[3] - b[3]) <= 1e-14 * a[3]


def test_fused_runs_to_time(hw):
    """Whole runs: the smooth periodic Euler problem, Example 3.8 (2D Burgers,
    smooth) and a shocked Burgers run past the shock time."""
    for w, tol in ((W.euler2d_smooth(32, t_end=0.2), 1e-10),
                   (W.burgers2d_sine(40), 1e-10),
                   (W.burgers2d_sine(40, t_end=1.5 / math.pi, dt_mode="cfl"), 1e-8)):
        g, _ = gpu_steps(hw, w, None, w.t_end, fused_2d=1)
        U, V, Wd, t, _ = O.run(oracle_problem(w), w.U, w.V, w.W, 0.0, w.t_end)
        check(w, g, (U, V, Wd, t), tol, tol)


def test_fused_double_mach_shocked_run(hw):
    w = W.double_mach(96, 24, t_end=0.02)
    g, _ = gpu_steps(hw, w, None, w.t_end, fused_2d=1)
    U, V, Wd, t, _ = O.run(oracle_problem(w), w.U, w.V, w.W, 0.0, w.t_end)
    check(w, g, (U, V, Wd, t), 1e-8, 1e-8)


@pytest.mark.parametrize("w", [W.euler2d_smooth(32, t_end=0.2), W.double_mach(96, 24, t_end=0.02)],
                         ids=["smooth", "double_mach"])
def test_fused_fp32_error(hw, w):
    """FP32 fused: the relative L-inf error against the FP64 oracle is as
    small as the split FP32 form's (within a factor of two of it, and
    under 1e-4)."""
    U, _, _, _, _ = O.run(oracle_problem(w), w.U, w.V, w.W, 0.0, w.t_end)
    shp = U.shape
    gs, _ = gpu_steps(hw, w, None, w.t_end, precision="fp32", fused_2d=0)
    gf, _ = gpu_steps(hw, w, None, w.t_end, precision="fp32", fused_2d=1)
    es, ef = rel(gs[0], U, shp), rel(gf[0], U, shp)
    assert ef <= 1e-4 and ef <= 2 * es + 1e-6, (ef, es)
    assert abs(gf[3] - gs[3]) <= 1e-6 * w.t_end


def test_fused_fp32_boundaries(hw):
    """FP32 fused, two steps with every boundary kind: the error against the
    FP64 oracle is within a factor of two of the split FP32 form's."""
    for bc in BCS:
        w = make_w("euler", 125, 8, bc, 21)
        gf, launches = gpu_steps(hw, w, 2, 1.0, precision="fp32", fused_2d=1)
        gs, _ = gpu_steps(hw, w, 2, 1.0, precision="fp32", fused_2d=0)
        assert launches == [5, 5]
        U, _, _, _, _ = O.run(oracle_problem(w), w.U, w.V, w.W, 0.0, 1.0, max_steps=2)
        es, ef = rel(gs[0], U, U.shape), rel(gf[0], U, U.shape)
        assert ef <= 1e-4 and ef <= max(2 * es, 1e-6), (bc, ef, es)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_autotune_chooses_a_form(hw, precision):
    """hweno_autotune in 2D times both forms of a stage, keeps the faster and
    the next step uses it (8 launches split, 5 fused)."""
    w = W.euler2d_smooth(256)
    s = hw.Solver.from_workload(w, precision=precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    U, V, Wd = dev(w.U, dt), dev(w.V, dt), dev(w.W, dt)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    U0 = U.clone()
    chosen, ms = s.autotune(U, V, Wd, t, 1.0)
    assert chosen in (0, 1)
    assert ms[0] > 0 and ms[1] > 0
    assert (ms[1] < ms[0]) == (chosen == 1)
    assert torch.equal(U, U0)  # tuning leaves the state alone
    s.step(U, V, Wd, t, 1.0)
    assert s.launches_last_call == (5 if chosen else 8)
    s.sync_status()
    s.close()


def test_options_reject_bad_fused_2d(hw):
    w = make_w("euler", 31, 50, BCS[0], 1)
    s = hw.Solver.from_workload(w)
    with pytest.raises(hw.HwenoError):
        s.set_options(fused_2d=2)
    s.close()


@pytest.mark.parametrize("fused", [0, 1])
def test_recorded_adjoint_replay_bits(hw, fused):
    """The adjoint of one step, with the stage states replayed in the same
    form as the forward step, gives the bits of the adjoint from a record of
    that step."""
    w = W.euler2d_smooth(40, ny=23, t_end=1.0)
    s = hw.Solver.from_workload(w, fused_2d=fused)
    U, V, Wd = dev(w.U), dev(w.V), dev(w.W)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    s.step(U, V, Wd, t, 1.0)
    U0, V0, W0, t0 = U.clone(), V.clone(), Wd.clone(), t.clone()
    dt = torch.empty(1, dtype=torch.float64, device="cuda")
    rec = s.new_record()
    s.step_record(U, V, Wd, t, 1.0, rec, dt)
    rng = np.random.default_rng(5)
    lam = [torch.from_numpy(rng.standard_normal(w.U.size)).cuda() for _ in range(3)]
    a = [x.clone() for x in lam]
    b = [x.clone() for x in lam]
    s.adjoint_step(U0, V0, W0, dt, *a, t=t0)
    assert s.launches_last_call == (9 if fused else 11)
    s.adjoint_step(U0, V0, W0, dt, *b, t=t0, record=rec)
    assert s.launches_last_call == 6
    s.sync_status()
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    s.close()


def test_options_keep_the_autotuned_form(hw):
    """hweno_get_options reports the stage form the autotuner chose, and
    set_options changes only the named options."""
    w = W.euler2d_smooth(64, t_end=1.0)
    s = hw.Solver.from_workload(w, dt_mode=1)
    U, V, Wd = dev(w.U), dev(w.V), dev(w.W)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    chosen, _ = s.autotune(U, V, Wd, t, 1.0)
    assert s.options().fused_2d == chosen
    s.set_options(cfl=0.3)
    o = s.options()
    assert o.fused_2d == chosen and o.dt_mode == 1 and o.cfl == 0.3
    s.set_options(fused_2d=1 - chosen)
    assert s.options().fused_2d == 1 - chosen and s.options().cfl == 0.3
    s.step(U, V, Wd, t, 1.0)
    assert s.launches_last_call == (5 if chosen == 0 else 8)
    with pytest.raises(AttributeError):
        s.set_options(no_such_option=1)
    s.close()
