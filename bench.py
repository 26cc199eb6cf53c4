#!/usr/bin/env python
"""Benchmark of the L-HWENO hot path: M point-updates/s per SSP-RK3 step.

Workload (default): the ragged batch of 2048 1D Euler Riemann problems
(gamma = 1.4, outflow, x in [0, 1], N per instance drawn from
{200, 400, 800, 1600, 3200}, 2.54 M points, seeded), FP64. One step is one
hweno_step over the whole batch: wave-speed reduction, three fused stage
kernels (ghosts, splitting, characteristic HWENO fluxes, linear derivative
fluxes, differences, limiter, RK combination) and the time update. A
point-update is one grid point advanced through one full step; instances
that have reached t_end do not count.

Prints one JSON line (rank 0). Timing: W warm-up steps; then K steps recorded
into a CUDA graph (hweno_run) and timed as one replay with CUDA events on the
library's stream, barrier and synchronize on both sides, max over ranks. The
per-step working set (state and stage buffers) is larger than the 129 MB L2,
so no flush is needed inside the graph. A second pass of K plain steps, each
bracketed by events with a 256 MiB L2 flush between steps, gives the per-
kernel durations for the roofline (library events around each launch) and
the no-graph comparison. Under torchrun each rank runs its own seeded batch
(weak scaling, no collective on the data path).

--impl reference times the CPU oracle (the reference arm of this build) on a
bounded sample of the same workload on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpoint-updates/s per RK step"
# Algorithmic operations per grid point of one SSP-RK3 step (+ - * / sqrt count
# one; abs and max zero), counted by the oracle's op-counting scalar on the
# scheme as the paper states it (only operations whose values reach the
# result); tests/test_bench_host.py re-derives them.
ALGO_FLOPS_PER_POINT_STEP = {
    ("euler", 1): 4870.21,
    ("burgers", 1): 1198.05,
    ("buckley", 1): 1296.27,
    ("euler", 2): 14555.81,
    ("burgers", 2): 2484.84,
}
# Algorithmic operations per grid point of one adjoint step: the op count of
# the oracle's forward-mode (dual-number) step, values and tangents together,
# on the adjoint workloads; one reverse step computes the same
# Jacobian-vector arithmetic transposed, plus the forward values it needs.
ALGO_ADJOINT_FLOPS_PER_POINT_STEP = {
    ("euler", 2): 45603.16,
    ("burgers", 1): 3722.17,
}
# Compulsory state traffic per point-step and component (words): 1D reads
# U^n,V^n / U1,V1,U^n,V~^n / U2,V2,U^n,V~^n and writes U1,V1,V~^n / U2,V2 /
# U^{n+1},V^{n+1}: 10 + 7 = 17.
ALGO_WORDS_PER_COMPONENT = {1: 17, 2: 26}
# ALU peaks (the recipe's nominal figures; no FP64/FP32 entry is measured in
# MEASURED_PEAKS.json): FP64 1.25 TFLOP/s; FP32 152 SMs x 128 lanes x 2 flop
# x 2.07 GHz.
PEAK_TFLOPS = {"fp64": 1.25, "fp32": 152 * 128 * 2 * 2.07e9 / 1e12}
# DRAM traffic constants from ncu captures (dram__bytes_read.sum +
# dram__bytes_write.sum of one launch over the points it processed) on cases
# whose working set exceeds the 129 MB L2; the bench scales them by the
# points of its own launch. An entry is set to None whenever its kernel
# changes after the capture (profiles/ holds the commands and the raw
# figures).
# Stage kernel, per point and launch (FP32: the 2048-instance batch, the
# mean of the three stage launches of one step of the autotuned tile).
MEASURED_STAGE_TRAFFIC_PER_POINT = {"fp64": None, "fp32": 52.5}
# Persistent kernel, per point-step (all three stages; FP64: 1024 instances,
# 1 283 400 points, one launch of 2 steps of the autotuned tile).
MEASURED_RUN_TRAFFIC_PER_POINT_STEP = {"fp64": 394.3, "fp32": None}
# One 2D stage per point, per workload, precision and stage form (0: the
# x-sweep + y-sweep launches of stage 1, 1: the fused stage-1 launch; smooth
# Euler at 1024^2, double Mach at 1920x480); applied to grids whose working
# set exceeds the L2.
MEASURED_STAGE_TRAFFIC_2D_PER_POINT = {("euler2d_smooth", "fp64", 0): 504.1,
                                       ("euler2d_smooth", "fp32", 0): 222.3,
                                       ("euler2d_smooth", "fp64", 1): 210.7,
                                       ("euler2d_smooth", "fp32", 1): 89.7,
                                       ("double_mach", "fp64", 0): 489.6}
# One 2D Euler adjoint step (six reverse sweeps, 128-thread CTAs) per point, 512^2.
MEASURED_ADJOINT_TRAFFIC_PER_POINT_STEP = {("euler", 2): 1862.6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "fp32"], default="fp64")
    ap.add_argument("--instances", type=int, default=2048)
    ap.add_argument("--workload", default="riemann_batch",
                    help="riemann_batch (default) | burgers1d:N | buckley_batch:COUNT | "
                         "euler2d_smooth:N | "
                         "double_mach:NXxNY | "
                         "burgers_adjoint:COUNTxN | euler2d_adjoint:N (discrete adjoint of the "
                         "step; own JSON line)")
    ap.add_argument("--fd-directions", type=int, default=16,
                    help="adjoint workloads: seeded directions checked by central differences")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the e2e, fp32 and cpu_baseline legs and the other workloads")
    ap.add_argument("--stage-2d", choices=["auto", "split", "fused"], default="auto",
                    help="2D stage form: auto (hweno_autotune times both and keeps the "
                         "faster), split (x-sweep + y-sweep launches) or fused (one launch)")
    ap.add_argument("--adjoint-steps-only", dest="light", action="store_true",
                    help="adjoint workloads: time the adjoint steps only (no full gradient, "
                         "no finite-difference checks)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = [r for r in self.rows if len(r) >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def rank_seed(rank: int) -> int:
    """Seed of the batch a rank runs (each rank its own batch: weak scaling)."""
    return 20220711 + rank


def reduce_over_ranks(ms: float, point_updates: float, device) -> tuple:
    """Job time = max over ranks; job work = sum over ranks."""
    import torch
    import torch.distributed as dist
    tt = torch.tensor([ms, point_updates], dtype=torch.float64, device=device)
    mx, sm = tt.clone(), tt.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1])


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def make_workload(name, rank, instances):
    """The benchmark workload `name` for a rank (see --workload)."""
    from paper_2207_05258_gb300 import workloads as W
    if name == "riemann_batch":
        return W.riemann_batch(count=instances, seed=rank_seed(rank))
    kind, _, size = name.partition(":")
    if kind == "burgers1d":
        return W.burgers1d_sine(int(size or 400))
    if kind == "buckley_batch":
        return W.buckley_batch(count=int(size or instances), seed=rank_seed(rank) + 1)
    if kind == "euler2d_smooth":
        return W.euler2d_smooth(int(size or 2048), dt_mode="cfl")
    if kind == "double_mach":
        nx, ny = (int(v) for v in (size or "1920x480").split("x"))
        return W.double_mach(nx, ny)
    raise SystemExit("unknown workload %r" % name)


def describe(w):
    if w.name == "buckley_batch":
        return ("buckley_batch: %d x Example 3.4 (Buckley-Leverett, u0 = 1 on [-1/2, 0]), "
                "N in {200,400,800,1600,3200}, %d points, t_end 0.4, outflow"
                % (w.batch, w.points))
    if w.name == "burgers1d_sine":
        return ("burgers1d: 1D Burgers periodic [0,2], N=%d, u0 = 0.5 + sin(pi x), "
                "T = 1.5/pi" % w.nx[0])
    if w.name == "riemann_batch":
        return ("riemann_batch: %d x 1D Euler Riemann problems, N in {200,400,800,1600,3200}, "
                "%d points, t_end 0.15, outflow" % (w.batch, w.points))
    if w.name == "euler2d_smooth":
        return ("euler2d_smooth: 2D Euler periodic [0,2]^2, rho = 1 + 0.2 sin(pi(x+y)), "
                "u = 0.7, v = 0.3, p = 1, %dx%d" % (w.nx[0], w.ny))
    return ("double_mach: Mach 10 shock at 60 deg on a wall, [0,4]x[0,1], %dx%d, t_end 0.2"
            % (w.nx[0], w.ny))


def _r4(x):
    return None if x is None else round(x, 4)


def scaled_traffic(table, key, units):
    """DRAM bytes of a launch from a per-unit table entry (None where the
    entry is missing or not captured for the kernel as it stands)."""
    per = table.get(key)
    return None if per is None else per * units


def traffic32(w, small, form, pts):
    """DRAM bytes of one FP32 stage launch (None where not captured)."""
    per = (MEASURED_STAGE_TRAFFIC_PER_POINT["fp32"] if w.dim == 1 and w.name == "riemann_batch"
           else MEASURED_STAGE_TRAFFIC_2D_PER_POINT.get((w.name, "fp32", form))
           if w.dim == 2 and not small else None)
    return None if per is None else per * pts


def working_set_mb(w, precision):
    """State plus library stage buffers touched by one step."""
    fields = 2 + 5 if w.dim == 1 else 3 + 8 + 4  # 2D adds W and the x-sweep scratch
    return fields * w.m * w.points * (8 if precision == "fp64" else 4) / 1e6


def run_ours(args, rank, world, dev_index):
    import torch
    from paper_2207_05258_gb300 import hweno

    torch.cuda.set_device(dev_index)
    w = make_workload(args.workload, rank, args.instances)
    nx = torch.tensor(w.nx if w.dim == 1 else [w.points], dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timed(precision, K, Wm, profile):
        """(a) K steps as one replay of a recorded CUDA graph (the headline);
        (b) with profile, K more plain steps, each bracketed by CUDA events with
        the kernels timed by the library's events and an L2 flush between
        steps (roofline and the no-graph comparison)."""
        force = (None if w.dim == 1 or args.stage_2d == "auto"
                 else int(args.stage_2d == "fused"))
        s = hweno.Solver.from_workload(w, precision=precision,
                                       **({} if force is None else {"fused_2d": force}))
        dt_t = torch.float64 if precision == "fp64" else torch.float32
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            U = torch.from_numpy(w.U).to("cuda", dt_t)
            V = torch.from_numpy(w.V).to("cuda", dt_t)
            Wd = torch.from_numpy(w.W).to("cuda", dt_t) if w.dim == 2 else None
            t = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
            hist = torch.zeros(K, w.batch, dtype=torch.float64, device="cuda")
            for _ in range(Wm):
                s.step(U, V, Wd, t, w.t_end)
            s.sync_status()
            # 1D: the tile shape; 2D: the split or the fused stage form (reads the
            # state only)
            tune = (s.autotune(U, V, Wd, t, w.t_end) if force is None
                    else (force, [None, None]))
            s.run_graph(U, V, Wd, t, w.t_end, max_steps=0, steps_per_launch=K)  # record
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if world > 1:
                import torch.distributed as dist
                dist.barrier()
            torch.cuda.synchronize()
            e0.record()
            steps, pu = s.run_graph(U, V, Wd, t, w.t_end, max_steps=K, steps_per_launch=K)
            e1.record()
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            ms = e0.elapsed_time(e1)
            launches = s.launches_last_call
            pers = None
            if w.dim == 1:  # the same K steps as one persistent launch
                p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s.run_persistent(U, V, t, w.t_end, 1)  # first call: scratch, occupancy
                if world > 1:
                    dist.barrier()
                torch.cuda.synchronize()
                s.profile_start(4)
                p0.record()
                ppu = s.run_persistent(U, V, t, w.t_end, K)  # synchronises after the kernel
                p1.record()
                torch.cuda.synchronize()
                run_ms = s.profile_read()["stage"][0]  # the persistent kernel alone
                pers = (p0.elapsed_time(p1), float(ppu), s.launches_last_call, run_ms)
                # the next K steps as that persistent launch recorded into a CUDA graph
                # and replayed; its point-updates are those of the same steps run
                # uncaptured on a copy of the state (the steps are deterministic)
                s.profile_start(0)
                Uc, Vc, tc = U.clone(), V.clone(), t.clone()
                gpu_ref = s.run_persistent(Uc, Vc, tc, w.t_end, K)
                del Uc, Vc
                cg = torch.cuda.CUDAGraph()
                with torch.cuda.graph(cg, capture_error_mode="thread_local"):
                    s.run_persistent(U, V, t, w.t_end, K, count=False)
                g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                if world > 1:
                    dist.barrier()
                torch.cuda.synchronize()
                g0.record()
                cg.replay()
                g1.record()
                torch.cuda.synchronize()
                s.sync_status()
                assert torch.equal(t, tc), "graph replay and direct run took different steps"
                del tc
                timed.pgraph = (g0.elapsed_time(g1), float(gpu_ref), 2)
            cls = None
            if w.dim == 1 and w.batch > 1 and profile:
                # tile variant per instance-size class, against the single variant
                chosen, cms = s.autotune_classes(U, V, t, w.t_end)
                cls = {"classes": s.size_classes(), "chosen": chosen,
                       "stage1_ms": [[round(x, 4) for x in row] for row in cms],
                       "stage1_ms_sum_single_variant": round(sum(r[tune[0]] for r in cms), 4),
                       "stage1_ms_sum_per_class": round(sum(min(r) for r in cms), 4),
                       "mixed_graph": None}
                if len(set(chosen)) > 1:  # the same K-step graph with per-class launches
                    s.run_graph(U, V, Wd, t, w.t_end, max_steps=0, steps_per_launch=K)
                    m0 = torch.cuda.Event(enable_timing=True)
                    m1 = torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    m0.record()
                    _, pum = s.run_graph(U, V, Wd, t, w.t_end, max_steps=K, steps_per_launch=K)
                    m1.record()
                    torch.cuda.synchronize()
                    mm = m0.elapsed_time(m1)
                    cls["mixed_graph"] = {"value": round(pum / (mm * 1e-3) / 1e6, 3),
                                          "ms_per_step": round(mm / K, 4),
                                          "launches_per_step": s.launches_last_call // K}
                s.set_class_variants([tune[0]] * len(chosen))  # back to one variant
            timed.cls = cls
            prof = ms_ng = pu_ng = None
            if profile:
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(K)]
                s.profile_start(K * 8 + 8)
                torch.cuda.synchronize()
                for i in range(K):
                    flush.zero_()
                    ev[i][0].record()
                    s.step(U, V, Wd, t, w.t_end, hist[i])
                    ev[i][1].record()
                torch.cuda.synchronize()
                s.sync_status()
                ms_ng = sum(a.elapsed_time(b) for a, b in ev)
                prof = s.profile_read()
                pu_ng = float(((hist > 0).double() * nx[None, :]).sum().item())
            clus = None
            if (profile and w.dim == 1 and max(w.nx) <= hweno.CLUSTER_MAX_POINTS and
                    working_set_mb(w, precision) < 129.0):
                # the same steps as one thread-block-cluster launch each
                # (fused_small = 2), timed the same way
                sc = hweno.Solver.from_workload(w, precision=precision, fused_small=2)
                for _ in range(Wm):
                    sc.step(U, V, Wd, t, w.t_end)
                sc.sync_status()
                evc = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                       for _ in range(K)]
                histc = torch.zeros(K, w.batch, dtype=torch.float64, device="cuda")
                sc.profile_start(K + 8)
                torch.cuda.synchronize()
                for i in range(K):
                    flush.zero_()
                    evc[i][0].record()
                    sc.step(U, V, Wd, t, w.t_end, histc[i])
                    evc[i][1].record()
                torch.cuda.synchronize()
                sc.sync_status()
                kern = sc.profile_read()["stage"]
                clus = (sum(a.elapsed_time(b) for a, b in evc),
                        float(((histc > 0).double() * nx[None, :]).sum().item()),
                        sc.launches_last_call * K, kern[0])
                # and the next K steps as one cluster launch (hweno_run_persistent),
                # L2 flushed before it; the events also cover the read-back of
                # the point-update count
                q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                flush.zero_()
                torch.cuda.synchronize()
                q0.record()
                cpu = sc.run_persistent(U, V, t, w.t_end, K)
                q1.record()
                torch.cuda.synchronize()
                timed.clus_run = (q0.elapsed_time(q1), float(cpu))
                sc.close()
        s.close()
        timed.tune = tune
        timed.pers = pers
        if pers is None:
            timed.pgraph = None
        timed.clus = clus
        if clus is None:
            timed.clus_run = None
        return ms, float(pu), prof, launches, ms_ng, pu_ng

    with ClockSampler(dev_index) as clk:
        ms, pu, prof, launches, ms_ng, pu_ng = timed(args.precision, args.steps, args.warmup, True)
    # the FP64 rate a DFMA-only loop reaches here (context for the FP64 roofline)
    fp64_loop = hweno.measure_fp64_peak() if args.precision == "fp64" else None
    clocks = clk.summary()
    tune = timed.tune
    pers = timed.pers
    clus = timed.clus

    # A working set that fits in L2 is timed step by step with an L2 flush
    # between steps (the plain pass); otherwise the graph replay is the
    # headline and the plain pass the comparison.
    small = working_set_mb(w, args.precision) < 129.0
    graph = {"value": round(pu / (ms * 1e-3) / 1e6, 3), "ms_per_step": round(ms / args.steps, 4),
             "note": "K steps as one CUDA-graph replay, no flush between steps"}
    plain = {"value": round(pu_ng / (ms_ng * 1e-3) / 1e6, 3),
             "ms_per_step": round(ms_ng / args.steps, 4),
             "note": "same steps launched one by one, L2 flushed between steps"}
    persistent = None
    pgraph = getattr(timed, "pgraph", None)
    if pers is not None:
        persistent = {"value": round(pers[1] / (pers[0] * 1e-3) / 1e6, 3),
                      "ms_per_step": round(pers[0] / args.steps, 4),
                      "note": "the next K steps as one persistent launch (hweno_run_persistent)"}
        if pgraph is not None:
            persistent["graph_replay"] = {
                "value": round(pgraph[1] / (pgraph[0] * 1e-3) / 1e6, 3),
                "ms_per_step": round(pgraph[0] / args.steps, 4),
                "note": "the next K steps: that persistent launch recorded into a CUDA graph "
                        "and replayed"}
    use_pers = (not small and pers is not None and pers[1] > 0 and
                pers[1] / pers[0] > pu / ms)
    timing_note = "K steps = one CUDA-graph replay (hweno_run), CUDA events"
    cluster = None
    if clus is not None:
        cluster = {"value": round(clus[1] / (clus[0] * 1e-3) / 1e6, 3),
                   "ms_per_step": round(clus[0] / args.steps, 4),
                   "note": "each step one launch on thread-block clusters (fused_small = 2), "
                           "L2 flushed between steps"}
    cluster_run = None
    if getattr(timed, "clus_run", None) and timed.clus_run[1] > 0:
        cr = timed.clus_run
        cluster_run = {"value": round(cr[1] / (cr[0] * 1e-3) / 1e6, 3),
                       "ms_per_step": round(cr[0] / args.steps, 4),
                       "note": "the next K steps as one launch on thread-block clusters "
                               "(hweno_run_persistent with fused_small = 2), L2 flushed "
                               "before the launch"}
    use_clus = (small and clus is not None and clus[1] > 0 and
                clus[1] / clus[0] > pu_ng / ms_ng)
    # small instances: the K steps in one cluster launch are the headline
    # where they beat one launch per step
    use_crun = (small and cluster_run is not None and use_clus and
                timed.clus_run[1] / timed.clus_run[0] > clus[1] / clus[0])
    if small:
        ms, pu = ms_ng, pu_ng
    if use_crun:
        ms, pu, launches = timed.clus_run[0], timed.clus_run[1], 1
    elif use_clus:
        ms, pu, launches = clus[0], clus[1], clus[2]
    elif use_pers and pgraph is not None:
        ms, pu, launches = pgraph[0], pgraph[1], pgraph[2]
        timing_note = ("K steps = one persistent launch (hweno_run_persistent) after one "
                       "wave-speed launch, recorded into a CUDA graph and replayed; CUDA events "
                       "around the replay")
    elif use_pers:
        ms, pu, launches = pers[0], pers[1], pers[2]
        timing_note = ("K steps = one persistent launch (hweno_run_persistent) after one "
                       "wave-speed launch, CUDA events")
    if world > 1:
        ms, pu = reduce_over_ranks(ms, pu, "cuda")
    value = pu / (ms * 1e-3) / 1e6

    # roofline of the dominant kernel (the fused stage kernel)
    stage_ms, stage_n = prof["stage"]
    pts_per_stage = pu_ng / args.steps  # points per stage in the profiled pass (this rank)
    flop_stage = ALGO_FLOPS_PER_POINT_STEP[(w.equation, w.dim)] / 3.0
    # a split 2D stage is two launches (x- and y-sweep), a fused one is one
    fused2d = w.dim == 2 and tune[0] == 1
    launches_per_stage = 1 if (w.dim == 1 or fused2d) else 2
    stage_time = stage_ms / stage_n * launches_per_stage * 1e-3
    achieved = flop_stage * pts_per_stage / stage_time / 1e12
    peak = PEAK_TFLOPS[args.precision]
    traffic = (MEASURED_STAGE_TRAFFIC_PER_POINT.get(args.precision)
               if args.workload == "riemann_batch" else
               MEASURED_STAGE_TRAFFIC_2D_PER_POINT.get((w.name, args.precision, tune[0]))
               if w.dim == 2 and not small
               else None)  # None: not captured for this workload
    if use_crun:  # the headline kernel: K steps in one cluster launch
        achieved = ALGO_FLOPS_PER_POINT_STEP[(w.equation, w.dim)] * pu / (ms * 1e-3) / 1e12
    elif use_clus:  # the headline kernel: one cluster launch per step
        achieved = ALGO_FLOPS_PER_POINT_STEP[(w.equation, w.dim)] * clus[1] / (clus[3] * 1e-3) / 1e12
    if use_pers:  # the headline kernel: K steps in one persistent launch
        run_s = pers[3] * 1e-3
        achieved = ALGO_FLOPS_PER_POINT_STEP[(w.equation, w.dim)] * pers[1] / run_s / 1e12
        rtraffic = MEASURED_RUN_TRAFFIC_PER_POINT_STEP.get(args.precision)
    roof = {"bound": "alu", "achieved": round(achieved, 4), "peak": peak, "unit": "TFLOP/s",
            "frac": round(achieved / peak, 4),
            **({"dfma_loop_tflops": round(fp64_loop, 4),
                "frac_of_dfma_loop": round(achieved / fp64_loop, 4)}
               if args.precision == "fp64" and fp64_loop else {}),
            "traffic": (None if traffic is None else traffic * pts_per_stage) if not use_pers else
                       (None if rtraffic is None else rtraffic * pers[1]),
            "kernel": ("k_run_1d<%s,%s> (K = %d steps per launch)" % (w.equation, args.precision,
                                                                     args.steps) if use_pers else
                       "%s<%s,%s>%s" % ("k_step_cluster_split_1d" if max(w.nx) <= 448 else
                                        "k_step_cluster_1d", w.equation, args.precision,
                                        " (K = %d steps per launch)" % args.steps
                                        if use_crun else "") if use_clus else
                       "k_stage_1d<%s,%s>" % (w.equation, args.precision) if w.dim == 1 else
                       "k_stage_2d<%s,%s> (fused x and y parts)" % (w.equation, args.precision)
                       if fused2d else
                       "k_xsweep_2d + k_ysweep_2d <%s,%s>" % (w.equation, args.precision)),
            "kernel_share_of_step": (round(pers[3] / pers[0], 4) if use_pers else
                                     1.0 if use_crun else
                                     round(clus[3] / clus[0], 4) if use_clus else
                                     round(stage_ms / sum(v[0] for v in prof.values()), 4)),
            "flops_per_point_stage": round(flop_stage, 2),
            "peak_source": "nominal (recipe): FP64 1.25 TFLOP/s; FP32 = 152 SM x 128 x 2 x 2.07 GHz",
            "hbm_achieved_gbs": round(ALGO_WORDS_PER_COMPONENT[w.dim] * w.m *
                                      (8 if args.precision == "fp64" else 4) *
                                      (pers[1] / (pers[3] * 1e-3) if use_pers else
                                       pu / (ms * 1e-3) if use_crun else
                                       clus[1] / (clus[3] * 1e-3) if use_clus else
                                       pts_per_stage / 3.0 / stage_time) / 1e9, 1)}

    out = {"metric": METRIC, "value": round(value, 3), "unit": "Mpoint-updates/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
           "us_per_step": round(ms / args.steps * 1e3, 2),
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic",
           ("graph" if small else "no_graph"): graph if small else plain,
           **({"graph": graph, "persistent": persistent} if use_pers else
              ({"persistent": persistent} if persistent else {})),
           **({"cluster": cluster} if cluster and (use_crun or not use_clus) else {}),
           **({"cluster_run": cluster_run} if cluster_run and not use_crun else {}),
           **({"plain": plain} if use_clus else {}),
           "config": {"workload": describe(w),
                      "instances": w.batch, "points": w.points, "precision": args.precision,
                      "l2": ("flushed before the timed launch (256 MiB write): the working "
                             "set (%.1f MB) fits in the 129 MB L2" % working_set_mb(w, args.precision)
                             if use_crun else
                             "flushed between timed steps (256 MiB write): the working set "
                             "(%.1f MB) fits in the 129 MB L2" % working_set_mb(w, args.precision)
                             if small else
                             "no flush inside the timed graph of K steps: the per-step working "
                             "set (state + stage buffers, %.0f MB) exceeds the 129 MB L2"
                             % (working_set_mb(w, args.precision))),
                      "timing": ("the K steps as one launch on thread-block clusters "
                                 "(hweno_run_persistent, fused_small = 2) after an L2 flush, "
                                 "CUDA events around the launch and the read-back of its "
                                 "point-update count" if use_crun else
                                 "each step (one launch on thread-block clusters, fused_small = 2) "
                                 "bracketed by CUDA events, summed over K steps" if use_clus else
                                 "each step bracketed by CUDA events, summed over K steps"
                                 if small else timing_note),
                      "tile_variant": tune[0] if w.dim == 1 else None,
                      "size_classes": getattr(timed, "cls", None),
                      "autotune_stage1_ms": ([round(x, 4) for x in tune[1]] if w.dim == 1 else
                                             {"split": _r4(tune[1][0]),
                                              "fused": _r4(tune[1][1])}),
                      **({"stage_form_2d": ("fused" if fused2d else "split") +
                          (" (autotuned)" if args.stage_2d == "auto" else " (forced)")}
                         if w.dim == 2 else {}),
                      "parallelism": "replicas (one seeded batch per rank)"},
           "roofline": roof, "clocks": clocks, "gpu_launches": launches,
           "point_updates_timed": pu}

    if not args.no_extras:
        # FP32 variant of the same workload (state and reconstruction in FP32)
        if args.precision == "fp64":
            ms32, pu32, prof32, _, _, pu32_ng = timed("fp32", args.steps, args.warmup, True)
            f32 = w.dim == 2 and timed.tune[0] == 1  # the form chosen for FP32
            st32 = prof32["stage"][0] / prof32["stage"][1] * (1 if (w.dim == 1 or f32) else 2) * 1e-3
            ach32 = flop_stage * (pu32_ng / args.steps) / st32 / 1e12
            out["fp32"] = {"value": round(pu32 / (ms32 * 1e-3) / 1e6, 3),
                           **({"stage_form_2d": "fused" if f32 else "split",
                               "autotune_stage1_ms": {"split": _r4(timed.tune[1][0]),
                                                      "fused": _r4(timed.tune[1][1])}}
                              if w.dim == 2 else {}),
                           "ms_per_step": round(ms32 / args.steps, 4),
                           "stage_kernel_ms": round(prof32["stage"][0] / prof32["stage"][1], 4),
                           "roofline": {
                               "bound": "alu", "achieved": round(ach32, 4),
                               "peak": round(PEAK_TFLOPS["fp32"], 2), "unit": "TFLOP/s",
                               "frac": round(ach32 / PEAK_TFLOPS["fp32"], 4),
                               "traffic": traffic32(w, small, timed.tune[0], pu32_ng / args.steps),
                               "kernel": ("k_stage_1d<%s,fp32>" % w.equation if w.dim == 1 else
                                          "k_stage_2d<%s,fp32> (fused x and y parts)" % w.equation
                                          if f32 else
                                          "k_xsweep_2d + k_ysweep_2d <%s,fp32>" % w.equation),
                               "flops_per_point_stage": round(flop_stage, 2),
                               "peak_source": "unit counts (recipe): 152 SM x 128 FP32 lanes x "
                                              "2 flop x 2.07 GHz"}}
            p32 = timed.pers
            if p32 is not None and p32[1] > 0:  # the same K steps as one persistent launch
                out["fp32"]["persistent"] = {"value": round(p32[1] / (p32[0] * 1e-3) / 1e6, 3),
                                             "ms_per_step": round(p32[0] / args.steps, 4)}
            c32 = timed.clus_run
            if c32 is not None and c32[1] > 0:  # small instances: K steps in one cluster launch
                out["fp32"]["cluster_run"] = {"value": round(c32[1] / (c32[0] * 1e-3) / 1e6, 3),
                                              "ms_per_step": round(c32[0] / args.steps, 4)}
        out["e2e"] = run_e2e(args, w, hweno, torch)
        if rank == 0 and w.dim == 1:
            out["cpu_baseline"] = cpu_baseline(w, budget_s=16.0)
    return out, rank


def run_e2e(args, w, hweno, torch):
    """Same metric through the C ABI's host-buffer entry point: every step
    copies U, V, t from pinned host memory and the result back (in 1D the
    library pipelines the copies of instance chunks with their kernels)."""
    # small 1D instances take the cluster step, as in the device-side measurement
    small1d = (w.dim == 1 and max(w.nx) <= hweno.CLUSTER_MAX_POINTS and
               working_set_mb(w, args.precision) < 129.0)
    s = hweno.Solver.from_workload(w, precision=args.precision,
                                   **({"fused_small": 2} if small1d else {}))
    dt_t = torch.float64 if args.precision == "fp64" else torch.float32
    if w.dim == 1:  # the same tile shape as the device-side measurement
        Ud = torch.from_numpy(w.U).to("cuda", dt_t)
        Vd = torch.from_numpy(w.V).to("cuda", dt_t)
        s.autotune(Ud, Vd, None, torch.zeros(w.batch, dtype=torch.float64, device="cuda"),
                   w.t_end)
        del Ud, Vd
    U = torch.from_numpy(w.U).to(dt_t).pin_memory()
    V = torch.from_numpy(w.V).to(dt_t).pin_memory()
    Wd = torch.from_numpy(w.W).to(dt_t).pin_memory() if w.dim == 2 else None
    t = torch.zeros(w.batch, dtype=torch.float64).pin_memory()
    sizes = np.array(w.nx if w.dim == 1 else [w.points])
    for _ in range(2):
        s.step_host(U, V, Wd, t, w.t_end, 1)
    K = max(3, args.steps // 2)
    pts = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K):
        active = (t.numpy() < w.t_end)
        pts += int(np.sum(sizes[active]))
        s.step_host(U, V, Wd, t, w.t_end, 1)
    el = time.perf_counter() - t0
    s.close()
    b = (U.numel() + V.numel() + (Wd.numel() if Wd is not None else 0)) * U.element_size() \
        + t.numel() * 8
    return {"value": round(pts / el / 1e6, 3), "unit": "Mpoint-updates/s",
            "h2d_bytes_per_step": b, "d2h_bytes_per_step": b, "steps": K}


def _oracle_problems(w, ks):
    import oracle as O
    eq = dict(burgers=O.EQ_BURGERS, euler=O.EQ_EULER, buckley=O.EQ_BUCKLEY)[w.equation]
    bcs = {"outflow": O.BC_OUTFLOW, "periodic": O.BC_PERIODIC, "inflow": O.BC_INFLOW,
           "reflective": O.BC_REFLECTIVE}
    return [O.problem(eq, 1, w.nx[k], 1, w.x0, w.x1, gas_gamma=w.gas_gamma,
                      bc=(bcs[w.bc[0]], bcs[w.bc[1]]), inflow=w.inflow) for k in ks]


def _oracle_worker(job):
    """One host process of the CPU baseline: one oracle step of each of its
    instances, repeated for budget_s seconds; returns (points, seconds)."""
    w, ks, budget_s = job
    import oracle as O
    probs = _oracle_problems(w, ks)
    states = [w.instance(k) for k in ks]
    O.step(probs[0], states[0][0], states[0][1], None, 0.0, w.t_end)  # load + warm
    pts, t0 = 0, time.perf_counter()
    while True:
        for p, k, st in zip(probs, ks, states):
            O.step(p, st[0], st[1], None, 0.0, w.t_end)
            pts += w.nx[k]
        if time.perf_counter() - t0 >= budget_s:
            break
    return pts, time.perf_counter() - t0


def cpu_baseline(w, budget_s=12.0, sample=128, processes=None):
    """The oracle as it stands on the host cores, on a bounded sample: one
    SSP-RK3 step of the first `sample` instances, repeated for `budget_s`
    seconds, (a) in one thread and (b) split over one process per core
    (spawned, the oracle is single-threaded). The all-core figure is the
    reported value."""
    import multiprocessing as mp
    sample = min(sample, w.batch)
    ks = list(range(sample))
    pts1, el1 = _oracle_worker((w, ks, budget_s / 2))
    ncores = processes or os.cpu_count() or 1
    ncores = max(1, min(ncores, sample))
    jobs = [(w, ks[i::ncores], budget_s / 2) for i in range(ncores)]
    with mp.get_context("spawn").Pool(ncores) as pool:
        res = pool.map(_oracle_worker, jobs)
    allv = sum(r[0] for r in res) / max(r[1] for r in res) / 1e6
    return {"value": round(allv, 5), "unit": "Mpoint-updates/s", "cores": ncores,
            "kind": "oracle",
            "single_thread": round(pts1 / el1 / 1e6, 5),
            "sample": "one SSP-RK3 step of the first %d instances (%d points), repeated for "
                      "%.1f s in each of %d spawned processes (instances dealt round robin); "
                      "single_thread: the same on one core"
                      % (sample, sum(w.nx[:sample]), budget_s / 2, ncores)}


def run_adjoint(args, rank, world, dev_index):
    """Discrete adjoint of the SSP-RK3 step (hweno_adjoint_step).

    Workloads: burgers_adjoint:COUNTxN (default 256 x 800: 1D Burgers,
    periodic, u0 = 0.5 + sin(pi x) + a seeded 4-mode perturbation, T = 0.5/pi,
    J = sum u(T)^2 dx) and euler2d_adjoint:N (default 512: 2D Euler periodic,
    the density wave plus a seeded 4-mode perturbation, 400 fixed steps of
    T/400, T = 0.25, J = sum rho(T)^2 dx dy). Measured: (a) K adjoint steps,
    each the reverse of a forward step from its step record (the stage
    states saved by hweno_step_record; the path of the autograd Function),
    timed one by one with CUDA events, L2 flushed between steps, and the same
    steps replaying stages 1-2 instead (`replay`); the forward step alone for
    the ratio; (b) one full
    gradient through the checkpointed autograd Function (checkpoint every 20
    steps), host-timed; (c) --fd-directions seeded smooth directions d: the
    adjoint's <grad J, d> against central differences of the GPU forward
    (whose alpha is not frozen, so they agree to the alpha response)."""
    import torch
    from paper_2207_05258_gb300 import hweno, workloads as W
    from paper_2207_05258_gb300.adjoint import run_to_time

    torch.cuda.set_device(dev_index)
    kind, _, size = args.workload.partition(":")
    two = kind == "euler2d_adjoint"
    if two:
        n = int(size or 512)
        w = W.euler2d_adjoint(n, seed=7 + rank)
        s = hweno.Solver.from_workload(w, dt_mode=2, dt_fixed=w.meta["dt"])
        t_end, max_steps = 1e30, w.meta["steps"]  # the fixed dt never lands
        cell = ((w.x1 - w.x0) / n) ** 2
        npts = n * n
        desc = ("euler2d_adjoint: 2D Euler periodic [0,2]^2 %dx%d, rho = 1 + 0.2 sin(pi(x+y)) "
                "+ seeded 4-mode perturbation (0.05), u = 0.7, v = 0.3, p = 1, %d steps of "
                "dt = %.3g (T = %.3g)" % (n, n, max_steps, w.meta["dt"], w.t_end))
        jfun = lambda UT: (UT[:npts] ** 2).sum() * cell
    else:
        count, n = (int(v) for v in (size or "256x800").split("x"))
        w = W.burgers_adjoint_batch(count=count, n=n, seed=5 + rank)
        s = hweno.Solver.from_workload(w)
        t_end, max_steps = w.t_end, 1 << 30
        cell = (w.x1 - w.x0) / n
        npts = count * n
        desc = ("burgers_adjoint: %d x 1D Burgers N=%d, periodic [0,2], u0 = 0.5 + sin(pi x) "
                "+ seeded 4-mode perturbation, T = 0.5/pi" % (count, n))
        jfun = lambda UT: (UT * UT).sum() * cell
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    K, Wm = args.steps, args.warmup
    cuda = lambda a: torch.from_numpy(a).cuda() if a is not None else None
    stream = torch.cuda.Stream()
    with ClockSampler(dev_index) as clk, torch.cuda.stream(stream):
        U, V, Wd = cuda(w.U), cuda(w.V), cuda(w.W)
        t = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
        states, dts, fwd = [], [], []
        for k in range(Wm + K):
            states.append((U.clone(), V.clone(), Wd.clone() if two else None, t.clone()))
            dt = torch.empty(w.batch, dtype=torch.float64, device="cuda")
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            s.step(U, V, Wd, t, t_end, dt)
            e1.record()
            dts.append(dt)
            fwd.append((e0, e1))
        # the same steps again, untimed, saving their stage states (step records)
        recs = [s.new_record() for _ in range(Wm + K)]
        for k in range(Wm + K):
            Uc, Vc = states[k][0].clone(), states[k][1].clone()
            Wc = states[k][2].clone() if two else None
            s.step_record(Uc, Vc, Wc, states[k][3].clone(), t_end, recs[k])
        lam0 = [2.0 * U * cell, torch.zeros_like(V)] + ([torch.zeros_like(Wd)] if two else [])
        if two:
            lam0[0][npts:] = 0.0

        def adjoint_pass(recorded):
            lam = [x.clone() for x in lam0]
            ev = []
            for k in range(Wm + K - 1, -1, -1):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                s.adjoint_step(states[k][0], states[k][1], states[k][2], dts[k], lam[0], lam[1],
                               lam[2] if two else None, t=states[k][3],
                               record=recs[k] if recorded else None)
                e1.record()
                ev.append((e0, e1))
            return ev

        adj = adjoint_pass(True)  # the path of the autograd Function
        launches = s.launches_last_call
        adj_rp = adjoint_pass(False)  # replaying stages 1-2 inside the adjoint step
        torch.cuda.synchronize()
        s.sync_status()
        adj_ms = sum(a.elapsed_time(b) for a, b in adj[Wm:])  # skip the warm-up steps
        replay_ms = sum(a.elapsed_time(b) for a, b in adj_rp[Wm:])
        del recs
        fwd_ms = sum(a.elapsed_time(b) for a, b in fwd[Wm:])
        if two:
            active = float(K * npts)
        else:
            active = float(sum(float((d > 0).double().sum().item()) for d in dts[:K])) * n
        del states
        light = getattr(args, "light", False)
        g, fd, grad_s = None, [], None
    if not light:
        with ClockSampler(dev_index), torch.cuda.stream(stream):
            g, fd, grad_s = _adjoint_gradient_checks(args, w, s, two, n, npts, count if not two
                                                     else 1, t_end, max_steps, jfun, cuda,
                                                     rank, W, run_to_time, torch)
    if world > 1:
        adj_ms, active = reduce_over_ranks(adj_ms, active, "cuda")
    value = active / (adj_ms * 1e-3) / 1e6
    key = ("euler", 2) if two else ("burgers", 1)
    ach = ALGO_ADJOINT_FLOPS_PER_POINT_STEP[key] * active / (adj_ms * 1e-3) / 1e12
    fp64_loop = hweno.measure_fp64_peak()
    out = {"metric": "Mpoint-updates/s per adjoint RK step", "value": round(value, 3),
           "unit": "Mpoint-updates/s", "n_gpus": world, "steps": K, "warmup": Wm,
           "ms_per_step": round(adj_ms / K, 4), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": desc,
                      "l2": "flushed between timed steps (256 MiB write)",
                      "timing": "CUDA events around each hweno_adjoint_step"},
           "forward_ms_per_step": round(fwd_ms / K, 4),
           "adjoint_over_forward": round(adj_ms / fwd_ms, 3),
           "replay": {"ms_per_step": round(replay_ms / K, 4),
                      "note": "hweno_adjoint_step without a step record: stages 1-2 "
                              "replayed inside the adjoint step"},
           "roofline": {"bound": "alu", "achieved": round(ach, 4), "peak": PEAK_TFLOPS["fp64"],
                        "unit": "TFLOP/s", "frac": round(ach / PEAK_TFLOPS["fp64"], 4),
                        "dfma_loop_tflops": round(fp64_loop, 4),
                        "frac_of_dfma_loop": round(ach / fp64_loop, 4),
                        "traffic": scaled_traffic(MEASURED_ADJOINT_TRAFFIC_PER_POINT_STEP, key,
                                                  npts),
                        "kernel": "hweno_adjoint_step (reverse stages 3, 2, 1; %d launches)"
                                  % launches,
                        "flops_per_point_step": ALGO_ADJOINT_FLOPS_PER_POINT_STEP[key],
                        "flops_source": "op count of the oracle's dual-number step (values "
                                        "and tangents)",
                        "peak_source": "nominal (recipe): FP64 1.25 TFLOP/s"},
           "clocks": clk.summary(), "gpu_launches": launches * K}
    if grad_s is not None:
        out["full_gradient"] = {"seconds": round(grad_s, 3), "checkpoint_every": 20,
                                "note": "forward run + checkpointed backward, host-timed"}
    if fd:
        out["fd_check"] = {"directions": len(fd), "eps": 1e-6,
                           "max_rel_to_cs_scale": max(f["rel_to_cs_scale"] for f in fd),
                           "max_rel_to_dJ": max(abs(f["adjoint"] - f["fd"]) / abs(f["fd"])
                                                for f in fd),
                           "first": fd[0]}
    return out


def _adjoint_gradient_checks(args, w, s, two, n, npts, count, t_end, max_steps, jfun, cuda,
                             rank, W, run_to_time, torch):
    """(b) one full gradient through the checkpointed autograd Function,
    host-timed; (c) central differences along --fd-directions seeded smooth
    directions against the adjoint's <grad J, d>."""
    # (b) full gradient with checkpoints
    U0, V0 = cuda(w.U).requires_grad_(True), cuda(w.V).requires_grad_(True)
    W0 = cuda(w.W).requires_grad_(True) if two else None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = run_to_time(U0, V0, s, t_end, 20, max_steps=max_steps, W0=W0)
    J = jfun(out[0])
    J.backward()
    torch.cuda.synchronize()
    grad_s = time.perf_counter() - t0
    g = [U0.grad, V0.grad] + ([W0.grad] if two else [])
    # (c) central differences along seeded smooth directions
    fd = []
    rng = W.SplitMix64(1234 + rank)
    for _ in range(args.fd_directions):
        if two:  # a perturbation of the initial density alone (and its derivatives)
            f, fx, fy = W.fourier_2d(rng, n, n, 0.0, 2.0, 1e-2)
            z = np.zeros(3 * npts)
            d = [np.concatenate([g.ravel(), z]) for g in (f, fx, fy)]
        else:
            x = W.centers(0.0, 2.0, n)
            du = np.concatenate([1e-2 * np.sin(np.pi * x * (1 + int(rng.uniform(0, 4))) +
                                               rng.uniform(0, 6.3)) for _ in range(count)])
            d = [du, np.zeros_like(du)]
        dg = [cuda(x) for x in d]
        adj_dJ = float(sum((gi * di).sum().item() for gi, di in zip(g, dg)))
        scale = math.sqrt(sum(float((gi * gi).sum().item()) for gi in g) *
                          sum(float((di * di).sum().item()) for di in dg))
        eps = 1e-6
        Js = []
        for sg in (1.0, -1.0):
            Ue = cuda(w.U) + sg * eps * dg[0]
            Ve = cuda(w.V) + sg * eps * dg[1]
            We = cuda(w.W) + sg * eps * dg[2] if two else None
            te = torch.zeros(w.batch, dtype=torch.float64, device="cuda")
            s.run(Ue, Ve, We, te, t_end, max_steps=max_steps)
            Js.append(float(jfun(Ue).item()))
        fdv = (Js[0] - Js[1]) / (2 * eps)
        fd.append({"adjoint": adj_dJ, "fd": fdv,
                   "rel_to_cs_scale": abs(adj_dJ - fdv) / scale})
    return g, fd, grad_s


# ---------------------------------------------------------------------------
# reference arm: the oracle
# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return None
    from paper_2207_05258_gb300 import workloads as W
    import oracle as O
    w = W.riemann_batch(count=args.instances, seed=rank_seed(0))
    sample = 32
    bcs = {"outflow": O.BC_OUTFLOW}
    probs = [O.problem(O.EQ_EULER, 1, w.nx[k], 1, w.x0, w.x1, gas_gamma=w.gas_gamma,
                       bc=(bcs[w.bc[0]], bcs[w.bc[1]])) for k in range(sample)]
    st = [[*w.instance(k), 0.0] for k in range(sample)]

    def one_step():
        n = 0
        for k in range(sample):
            U, V, _, tk, _ = O.step(probs[k], st[k][0], st[k][1], None, st[k][2], w.t_end)
            st[k] = [U, V, tk]
            n += w.nx[k]
        return n

    for _ in range(args.warmup):
        one_step()
    pts, t0 = 0, time.perf_counter()
    for _ in range(args.steps):
        pts += one_step()
    el = time.perf_counter() - t0
    v = pts / el / 1e6
    pts_sample = sum(w.nx[:sample])
    return {"impl": "reference", "metric": METRIC, "value": round(v, 5),
            "unit": "Mpoint-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "riemann_batch: first %d of %d 1D Euler Riemann problems "
                                   "(%d points) per step" % (sample, w.batch, pts_sample),
                       "instances": sample, "points": pts_sample, "precision": "fp64"},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "value": round(v, 5),
                             "unit": "Mpoint-updates/s",
                             "sample": "one SSP-RK3 step of the first %d instances per timed step"
                                       % sample},
            "e2e": {"value": round(v, 5), "unit": "Mpoint-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


# The other workloads of the benchmark suite, each timed briefly in the same
# run and reported as a sub-object of the headline line (N = 1 only):
# (key, --workload, precisions, K, W)
OTHER_CONFIGS = (
    ("burgers1d_n400", "burgers1d:400", ("fp64",), 20, 5),
    ("euler2d_smooth_256", "euler2d_smooth:256", ("fp64", "fp32"), 20, 3),
    ("euler2d_smooth_512", "euler2d_smooth:512", ("fp64", "fp32"), 20, 3),
    ("euler2d_smooth_1024", "euler2d_smooth:1024", ("fp64", "fp32"), 10, 3),
    ("euler2d_smooth_2048", "euler2d_smooth:2048", ("fp64", "fp32"), 10, 3),
    ("double_mach_1920x480", "double_mach:1920x480", ("fp64", "fp32"), 20, 3),
    ("double_mach_3840x960", "double_mach:3840x960", ("fp64", "fp32"), 5, 2),
)


def _compact(out):
    keep = ("value", "unit", "ms_per_step", "us_per_step", "steps", "warmup", "dtype",
            "roofline", "clocks", "gpu_launches", "cluster", "cluster_run", "graph", "no_graph",
            "plain", "persistent", "forward_ms_per_step", "adjoint_over_forward", "replay")
    c = {k: out[k] for k in keep if k in out}
    cfg = out.get("config", {})
    c["workload"] = cfg.get("workload")
    for k in ("timing", "l2", "stage_form_2d", "autotune_stage1_ms"):
        if k in cfg and not (k == "autotune_stage1_ms" and isinstance(cfg[k], list)):
            c[k] = cfg[k]
    return c


def other_configs(args, dev_index):
    """The other benchmark workloads, each with its own roofline, for the
    headline line: 1D Burgers N = 400, the smooth 2D Euler grids 256^2 to
    2048^2 and the double Mach grids 1920 x 480 and 3840 x 960 (FP64 and
    FP32), and the adjoint steps of the 2D Euler 512^2 problem and of the
    batch of 256 Burgers problems with N = 800."""
    import copy
    res = {}
    # a failing sub-configuration is reported in its own entry and does not
    # take the headline line with it
    for key, wl, precs, K, Wm in OTHER_CONFIGS:
        for prec in precs:
            a = copy.copy(args)
            a.workload, a.precision, a.no_extras, a.steps, a.warmup = wl, prec, True, K, Wm
            try:
                out, _ = run_ours(a, 0, 1, dev_index)
                res.setdefault(key, {})[prec] = _compact(out)
            except Exception as e:  # noqa: BLE001
                res.setdefault(key, {})[prec] = {"error": repr(e)[:300]}
    for key, wl, K in (("euler2d_adjoint_512", "euler2d_adjoint:512", 5),
                       ("burgers_adjoint_256x800", "burgers_adjoint:256x800", 10)):
        a = copy.copy(args)
        a.workload, a.steps, a.warmup, a.fd_directions, a.light = wl, K, 2, 0, True
        try:
            res[key] = _compact(run_adjoint(a, 0, 1, dev_index))
        except Exception as e:  # noqa: BLE001
            res[key] = {"error": repr(e)[:300]}
    return res


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    if args.workload.startswith(("burgers_adjoint", "euler2d_adjoint")):
        out = run_adjoint(args, rank, world, local)
    else:
        out, rank = run_ours(args, rank, world, local)
        if world == 1 and not args.no_extras and args.workload == "riemann_batch":
            out["configs"] = other_configs(args, local)
            out["gpu_launches_configs"] = sum(
                v.get("gpu_launches", 0) for c in out["configs"].values()
                for v in (c.values() if "value" not in c else [c]))
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
