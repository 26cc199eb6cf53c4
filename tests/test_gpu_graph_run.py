"""hweno_run: steps recorded once into a CUDA graph and replayed until every
instance lands on t_end. The result must equal plain hweno_step calls bit for
bit (same kernels, same arguments; steps of finished instances are no-ops),
and the device point-update counter must equal sum_k N_k * steps_k with the
per-instance step counts of the oracle."""
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


def _subset(w, pick):
    Us, Vs = zip(*(w.instance(k) for k in pick))
    return W.Workload("sub", "euler", 1, [w.nx[k] for k in pick], 1, w.x0, w.x1, w.y0, w.y1,
                      w.t_end, w.bc, np.concatenate([u.ravel() for u in Us]),
                      np.concatenate([v.ravel() for v in Vs]))


@pytest.mark.parametrize("k", [1, 7, 32])
def test_graph_run_matches_plain_steps(hw, k):
    full = W.riemann_batch(count=40, seed=99)
    w = _subset(full, [i for i in range(40) if full.nx[i] <= 400][:8])
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = hw.Solver.from_workload(w)
        U, V = torch.from_numpy(w.U.copy()).cuda(), torch.from_numpy(w.V.copy()).cuda()
        t = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
        steps, pu = s.run_graph(U, V, None, t, w.t_end, steps_per_launch=k)
        s2 = hw.Solver.from_workload(w)
        U2, V2 = torch.from_numpy(w.U.copy()).cuda(), torch.from_numpy(w.V.copy()).cuda()
        t2 = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
        s2.run(U2, V2, None, t2, w.t_end, check_every=1)
    torch.cuda.synchronize()
    assert torch.equal(U, U2) and torch.equal(V, V2) and torch.equal(t, t2)
    assert torch.all(t == w.t_end)
    expect = 0
    for i in range(w.batch):
        Ui, Vi = w.instance(i)
        _, _, _, _, n = O.run(oracle_problem(w, nx=w.nx[i]), Ui, Vi, None, 0.0, w.t_end)
        expect += n * w.nx[i]
    assert pu == expect
    assert steps % k == 0 and steps >= max(1, pu // sum(w.nx))


def test_graph_run_2d_and_record_only(hw):
    w = W.double_mach(64, 16, t_end=0.01)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = hw.Solver.from_workload(w)
        U = torch.from_numpy(w.U.copy()).cuda()
        V, Wd = torch.zeros_like(U), torch.zeros_like(U)
        t = torch.zeros(1, dtype=torch.float64, device="cuda")
        steps, pu = s.run_graph(U, V, Wd, t, w.t_end, max_steps=0, steps_per_launch=4)
        assert steps == 0 and pu == 0 and float(t.item()) == 0.0
        steps, pu = s.run_graph(U, V, Wd, t, w.t_end, steps_per_launch=4)
    torch.cuda.synchronize()
    assert float(t.item()) == w.t_end
    U2, V2, W2, tt, n = O.run(oracle_problem(w), w.U, w.V, w.W, 0.0, w.t_end)
    assert pu == n * 64 * 16
    assert np.max(np.abs(U.cpu().numpy().reshape(U2.shape) - U2)) <= 1e-10 * np.max(np.abs(U2))


def test_graph_run_needs_a_stream(hw):
    w = W.burgers1d_sine(64)
    s = hw.Solver.from_workload(w)
    U, V = torch.from_numpy(w.U.copy()).cuda(), torch.from_numpy(w.V.copy()).cuda()
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    import ctypes
    rc = hw.lib.hweno_run(s.h, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(V.data_ptr()), None,
                          ctypes.c_void_p(t.data_ptr()), 1.0, 10, 4, None, None, None)
    assert rc == hw.EINVAL


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_every_tile_variant_gives_the_same_bits(hw, precision):
    """The tile shape only changes which CTA computes a point, not its
    arithmetic: all variants give the same state bits, and the autotuner picks
    the fastest."""
    full = W.riemann_batch(count=24, seed=17)
    w = full
    dt = torch.float64 if precision == "fp64" else torch.float32
    outs = []
    for v in range(hw.TILE_VARIANTS):
        s = hw.Solver.from_workload(w, precision=precision, tile_variant=v)
        U, V = torch.from_numpy(w.U).to("cuda", dt), torch.from_numpy(w.V).to("cuda", dt)
        t = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
        for _ in range(3):
            s.step(U, V, None, t, w.t_end)
        s.sync_status()
        outs.append((U.cpu(), V.cpu(), t.cpu(), s.totals(U).cpu()))
        s.close()
    for o in outs[1:]:
        for a, b in zip(outs[0][:3], o[:3]):
            assert torch.equal(a, b)
        # the totals' fixed summation order follows the tile size
        assert torch.allclose(outs[0][3], o[3], rtol=1e-14, atol=0)
    s = hw.Solver.from_workload(w, precision=precision)
    U, V = torch.from_numpy(w.U).to("cuda", dt), torch.from_numpy(w.V).to("cuda", dt)
    chosen, ms = s.autotune(U, V, None, torch.zeros(w.batch, dtype=torch.float64, device="cuda"),
                            w.t_end)
    assert 0 <= chosen < hw.TILE_VARIANTS and all(m > 0 for m in ms)
    assert ms[chosen] == min(ms)


def test_size_classes_of_the_riemann_batch(hw):
    full = W.riemann_batch(count=64, seed=3)
    s = hw.Solver.from_workload(full)
    assert s.size_classes() == [(n, n) for n in sorted(set(full.nx))]
    # more distinct sizes than classes: octaves above the smallest instance
    sizes = list(range(60, 60 + 40 * 9, 9))
    w = W.Workload("oct", "burgers", 1, sizes, 1, 0.0, 2.0, 0.0, 1.0, 1.0, ("periodic",) * 4,
                   np.ones(sum(sizes)), np.zeros(sum(sizes)))
    cl = hw.Solver.from_workload(w).size_classes()
    assert cl[0][0] == 60 and cl[-1][1] == max(sizes)
    assert all(lo <= hi for lo, hi in cl)
    assert all(cl[q][1] < cl[q + 1][0] for q in range(len(cl) - 1))
    assert [(lo, hi) for lo, hi in cl] == [(60, 114), (123, 231), (240, 411)]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mixed_tile_variants_per_size_class_give_the_same_bits(hw, precision):
    """Each size class on its own tile variant (one launch per class and
    stage): the state bits of a single variant, also through hweno_run's
    graph; hweno_autotune_classes picks the fastest variant per class."""
    w = W.riemann_batch(count=40, seed=17)
    dt = torch.float64 if precision == "fp64" else torch.float32
    nq = len(set(w.nx))

    def run(s, graph):
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            U, V = torch.from_numpy(w.U).to("cuda", dt), torch.from_numpy(w.V).to("cuda", dt)
            t = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
            if graph:
                s.run_graph(U, V, None, t, w.t_end, max_steps=3, steps_per_launch=3)
            else:
                for _ in range(3):
                    s.step(U, V, None, t, w.t_end)
        stream.synchronize()
        s.sync_status()
        return U.cpu(), V.cpu(), t.cpu()

    ref = run(hw.Solver.from_workload(w, precision=precision), False)
    mixed = hw.Solver.from_workload(w, precision=precision)
    mixed.set_class_variants([q % hw.TILE_VARIANTS for q in range(nq)])
    for graph in (False, True):
        out = run(mixed, graph)
        if not graph:
            assert mixed.launches_last_call == 2 + 3 * nq
        for a, b in zip(ref, out):
            assert torch.equal(a, b)
    s = hw.Solver.from_workload(w, precision=precision)
    U, V = torch.from_numpy(w.U).to("cuda", dt), torch.from_numpy(w.V).to("cuda", dt)
    chosen, ms = s.autotune_classes(U, V, None, w.t_end)
    assert len(chosen) == nq and all(0 <= v < hw.TILE_VARIANTS for v in chosen)
    for q in range(nq):
        assert ms[q][chosen[q]] == min(ms[q]) and all(m > 0 for m in ms[q])
    for a, b in zip(ref, run(s, False)):
        assert torch.equal(a, b)
    with pytest.raises(hw.HwenoError):
        s.set_class_variants([hw.TILE_VARIANTS] * nq)


def test_options_report_the_autotuned_tile_and_keep_the_rest(hw):
    """hweno_get_options after hweno_autotune holds the chosen tile variant;
    set_options(cfl=...) keeps it and the other options."""
    full = W.riemann_batch(count=16, seed=3)
    s = hw.Solver.from_workload(full, dt_mode=1, limiter=2)
    U, V = torch.from_numpy(full.U).cuda(), torch.from_numpy(full.V).cuda()
    t = torch.zeros(full.batch, dtype=torch.float64, device="cuda")
    chosen, _ = s.autotune(U, V, None, t, full.t_end)
    assert s.options().tile_variant == chosen
    s.set_options(cfl=0.4)
    o = s.options()
    assert (o.tile_variant, o.dt_mode, o.limiter, o.cfl) == (chosen, 1, 2, 0.4)
    assert list(o.lin_w) == [0.98, 0.01, 0.01]
    s.close()
