"""The JSON line bench.py prints: every key the benchmark contract asks for,
with the right types, for the reference arm (the CPU oracle, runs anywhere)
and for the GPU arm (a small render set, marked gpu)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
COMMON = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
          "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e",
          "cpu_baseline")


def _run(*args):
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, p.stdout
    return json.loads(lines[0])


def _check_common(d, steps, warmup):
    for k in COMMON:
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "rays/s" and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == steps and d["warmup"] == warmup
    assert d["scaling"] == "weak" and d["data"] == "synthetic" and d["dtype"] == "f64"
    assert d["vs_baseline"] is None  # the paper publishes no number for this workload
    assert isinstance(d["config"]["workload"], str) and d["config"]["workload"]
    e = d["e2e"]
    assert e["value"] > 0 and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] >= 0 and e["d2h_bytes_per_step"] >= 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] > 0 and cb["sample"]


def test_clock_summary_flags_throttling():
    """The clocks object: median SM clock under load, and every throttle
    reason that was Active in any sample (the contract rejects runs with
    hw_slowdown, hw_thermal_slowdown or sw_thermal_slowdown)."""
    sys.path.insert(0, ROOT)
    import bench
    idle = "0, 2070, 2070, 245.50, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1905, 2070, 1398.20, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
    hot = "0, 1500, 2070, 900.00, 0x0000000000000048, Active, Active, Not Active, Not Active"
    c = bench.summarize_clock_lines([idle, idle, capped, "garbage line", idle])
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0 and c["samples"] == 4
    assert c["reasons"] == ["sw_power_cap"] and c["power_w_max"] == 1398.2
    c = bench.summarize_clock_lines([hot, idle, hot])
    assert c["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"] and c["sm_mhz"] == 1500.0
    assert bench.summarize_clock_lines([])["reasons"] == ["no samples"]


def test_reference_arm_line():
    d = _run("--impl", "reference", "--side", "128", "--steps", "1", "--warmup", "1")
    _check_common(d, 1, 1)
    assert d["impl"] == "reference"
    assert d["cpu_baseline"]["value"] == d["value"] == d["e2e"]["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


@pytest.mark.parametrize("workload,name", [("qmetric", "qmetric_shadow"),
                                           ("disk_l0", "paper_disk_figure"),
                                           ("uneven", "uneven_batch"),
                                           ("timelike", "timelike")])
def test_reference_arm_next_workloads(workload, name):
    """The measured next rows through the same contract: the oracle with each
    render kind's options (q-metric, constant-l0 disk, mixed shadow/disk)."""
    d = _run("--impl", "reference", "--workload", workload, "--side", "32", "--steps", "1",
             "--warmup", "1")
    _check_common(d, 1, 1)
    assert d["config"]["workload"].startswith(name)
    assert "32" in d["config"]["workload"]


@pytest.mark.gpu
def test_gpu_arm_line():
    d = _run("--side", "64", "--steps", "1", "--warmup", "3", "--serve-seconds", "0.5",
             "--hbar-side", "32")
    _check_common(d, 1, 3)
    assert "impl" not in d or d["impl"] != "reference"
    r = d["roofline"]
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["peak"] > 0
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-9)
    assert "traffic" in r
    c = d["clocks"]
    assert c["sm_max_mhz"] > 0 and isinstance(c["reasons"], list)
    assert d["gpu_launches"] == 1  # one batched launch per timed step
    assert d["e2e"]["api"] == "osiris_batch_plan_launch"
    assert d["e2e"]["h2d_bytes_per_step"] > 0 and d["e2e"]["d2h_bytes_per_step"] > 0
    assert d["variants"]["df64"]["value"] > 0
    sv = d["serving"]
    assert sv["continuous_batching"]["p99_latency_s"] > 0
    assert "0.5 s" in sv["continuous_batching"]["workload"]
    assert "windows" in sv["continuous_batching"]
    assert isinstance(sv["continuous_batching"]["kept_up"], bool)
    assert sv["one_render_per_launch_fp64"]["renders"] > 0
    p = d["pipe_probes"]
    assert p["fp64_fma"]["tflops"] == pytest.approx(r["peak"], rel=1e-12)
    assert p["fp32_fma"]["tflops"] > p["fp64_fma"]["tflops"]
    hb = d["hbar"]
    assert hb["bar"] == 1e-10
    assert set(hb["ck45_tol1e-10"]["by_status"]) <= {"captured", "escaped", "disk"}
    assert len(hb["sweep"]["points"]) == 6
    assert d["other_configs"] is None  # the other configurations run only at the full size


@pytest.mark.gpu
@pytest.mark.parametrize("workload", ["qmetric", "disk_l0", "uneven", "timelike"])
def test_gpu_arm_next_workloads(workload):
    d = _run("--workload", workload, "--side", "32", "--steps", "1", "--warmup", "3",
             "--serve-seconds", "0.5")
    _check_common(d, 1, 3)
    assert d["metric"] != "rays/s (Kerr shadow+ring renders, FP64 Cash-Karp)"
    assert d["gpu_launches"] == 1
    assert d["roofline"]["f_rhs"] == (60 if workload == "qmetric" else 59)
    assert d["roofline"]["traffic"] is None
    assert d["variants"]["df64"]["value"] > 0
    assert d["serving"] is None  # the served stream is a Kerr workload
    if workload in ("disk_l0", "uneven"):
        assert d["status_counts_per_step"]["status_disk"] > 0
    if workload == "timelike":  # unbound particles launched outwards all escape
        assert d["status_counts_per_step"]["status_escaped"] == d["config"]["rays_per_step_per_gpu"]
        assert d["e2e"]["api"] == "osiris_trace_states_ex" and d["e2e"]["h2d_bytes_per_step"] > 0


def test_reference_arm_under_torchrun_two_ranks():
    """The driver's multi-rank launch of the reference arm: rank 0 alone times
    the oracle and prints one line; the other rank exits 0 without work."""
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    p = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
                        "--master-port", str(port), os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--side", "32", "--steps", "1", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, p.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def test_fp32_roofline_arithmetic():
    """The FP32-pipe roofline of DF64 and MIXED: FMA-pipe thread instructions
    per attempt x attempts/s over 32 x the probe's warp-instruction rate, and
    the issue fraction: warp instructions per attempt x attempts/s over the
    probe's warp-instruction rate (one per cycle per SM sub-partition)."""
    import bench
    probe = {"fp32_fma": {"warp_inst_per_s": 1.25e12}}
    r = bench.fp32_roofline(probe, 600, 40.0, attempts=3.0e9, seconds=0.1)
    assert r["peak"] == pytest.approx(1.25e12 * 32 / 1e12)
    assert r["achieved"] == pytest.approx(3.0e10 * 600 / 1e12)
    assert r["frac"] == pytest.approx(3.0e10 * 600 / (1.25e12 * 32))
    assert r["issue_frac"] == pytest.approx(3.0e10 * 40.0 / 1.25e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    # the constants in use: FMA-pipe instructions are a part of all those issued
    for ipa, wpa in ((bench.DF64_FP32_INST_PER_ATTEMPT, bench.DF64_WARP_INST_PER_ATTEMPT),
                     (bench.MIXED_FP32_INST_PER_ATTEMPT, bench.MIXED_WARP_INST_PER_ATTEMPT)):
        assert 0 < ipa < 32 * wpa


def test_workload_inputs():
    """Each workload's inputs: render counts and sizes, and the time-like
    particles on the mass shell H = -1/2 (the oracle's Kerr Hamiltonian),
    moving outwards."""
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    assert len(bench.workload_renders("kerr", 64)) == 12
    assert len(bench.workload_renders("qmetric", 64)) == 6
    assert all(rd["q"] is not None for rd in bench.workload_renders("qmetric", 64))
    l0 = bench.workload_renders("disk_l0", 64)
    assert len(l0) == 3 and all((rd["nx"], rd["ny"]) == (128, 64) for rd in l0)
    un = bench.workload_renders("uneven", 64)
    assert len(un) == 256 and {rd["nx"] for rd in un} <= {8, 16, 32, 64}
    assert bench.workload_renders("timelike", 64) == []
    st, E, L = bench.timelike_states(2000)
    assert st.shape == (E.size, 6) and E.size > 1900
    assert np.all(st[:, 4] > 0.0) and np.all(st[:, 5] == 0.0)
    for k in range(0, E.size, 97):
        H = oracle.hamiltonian(bench.TIMELIKE_A, st[k], E[k], L[k])
        assert abs(H + 0.5) < 1e-12, (k, H)
