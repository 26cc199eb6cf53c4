"""The bench's JSON line on small workloads: every key the measurement
contract asks for is present and consistent (value, ms per step, roofline
with its fraction, clocks, launches, e2e and cpu_baseline where they are
taken). Each case runs bench.py in a subprocess, as a user would."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def bench(*args, timeout=600):
    r = subprocess.run([sys.executable, "bench.py", *args], cwd=ROOT, capture_output=True,
                       text=True, timeout=timeout)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def check_common(d, steps, warmup):
    assert d["metric"] and d["unit"] == "Mpoint-updates/s"
    assert d["steps"] == steps and d["warmup"] == warmup and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert d["dtype"] in ("f64", "f32") and d["data"] == "synthetic"
    r = d["roofline"]
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["peak"] > 0
    assert r["achieved"] > 0 and abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-3
    assert r["traffic"] is None or r["traffic"] > 0
    assert d["gpu_launches"] >= 1
    c = d["clocks"]
    assert "sm_mhz" in c and "reasons" in c


def test_riemann_batch_line_with_every_leg():
    d = bench("--instances", "64", "--steps", "3", "--warmup", "3", "--precision", "fp64")
    check_common(d, 3, 3)
    # 64 instances fit in L2: timed step by step with a flush (the stage
    # kernel); batches larger than L2 take the persistent launch
    assert d["roofline"]["kernel"].startswith(("k_run_1d", "k_stage_1d"))
    assert d["roofline"]["dfma_loop_tflops"] > 0
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] > 0
    assert d["fp32"]["value"] > 0 and d["fp32"]["roofline"]["frac"] > 0
    assert "configs" in d  # the other workloads, each with its own line
    for k, v in d["configs"].items():
        entries = v.values() if ("fp64" in v or "fp32" in v) else [v]
        for x in entries:
            assert "error" not in x, (k, x)
            assert x["value"] > 0 and x["roofline"]["frac"] > 0, k


@pytest.mark.parametrize("form", ["split", "fused", "auto"])
def test_2d_line_reports_the_stage_form(form):
    d = bench("--workload", "euler2d_smooth:256", "--steps", "3", "--warmup", "3",
              "--no-extras", "--stage-2d", form)
    check_common(d, 3, 3)
    got = d["config"]["stage_form_2d"]
    if form != "auto":
        assert got == form + " (forced)"
        assert d["gpu_launches"] == 3 * (5 if form == "fused" else 8)
    else:
        ms = d["config"]["autotune_stage1_ms"]
        assert got.endswith("(autotuned)") and ms["split"] > 0 and ms["fused"] > 0
        assert got.startswith("fused" if ms["fused"] < ms["split"] else "split")


def test_small_instance_line_takes_the_cluster_launch():
    d = bench("--workload", "burgers1d:400", "--steps", "5", "--warmup", "3", "--no-extras")
    check_common(d, 5, 3)
    assert "k_step_cluster_split_1d" in d["roofline"]["kernel"]
    assert "cluster" in d or "cluster_run" in d


def test_adjoint_line():
    d = bench("--workload", "euler2d_adjoint:64", "--steps", "2", "--warmup", "1",
              "--fd-directions", "2", timeout=900)
    assert d["value"] > 0 and d["adjoint_over_forward"] > 1
    assert d["roofline"]["frac"] > 0
    assert d["fd_check"]["max_rel_to_cs_scale"] < 1e-6
