"""Benchmark: Kerr shadow / Einstein-ring renders, rays per second.

One step = one pass of the whole hot path (initial data, Cash-Karp
integration of Hamilton's equations, stopping surfaces, observables) over the
twelve 1024x1024 renders of the Kerr set: spin a in {0, 0.5, 0.9, 0.998} x
inclination in {17, 60, 90} deg, r_obs = 1000, image plane [-8, 8]^2,
tol 1e-10, seeded 10-degree checkerboard, FP64. By default the twelve renders
go through ONE persistent batched launch (osiris_trace_batch).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0). With N > 1 (torchrun) every rank renders its
own copy of the set (weak scaling) and the time is the max over ranks.
`--impl reference` times the CPU oracle (the only other implementation of the
method here) on a bounded pixel sample of the same workload.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD_NAME = ("kerr_shadow_ring: 12 renders (a in {0,0.5,0.9,0.998} x incl in {17,60,90} deg), "
                 "r_obs=1000, 1024x1024 cell centres on [-8,8]^2, Cash-Karp tol 1e-10, "
                 "r_cap=1.01 r_H, r_esc=1.1 r_obs, seeded 10-deg checkerboard")
METRIC = "rays/s (Kerr shadow+ring renders, FP64 Cash-Karp)"
UNIT = "rays/s"
# Algorithmic FP64 operations (FMA = 2, add/mul = 1, sincos and reciprocal = 1
# each) of one evaluation of the separated Hamilton equations, and of one
# Cash-Karp attempt besides its six evaluations (stage sums, fifth-order sum,
# error estimate, error norm, step clamp).
F_RHS = 59
F_STEP = 258
# The q-metric evaluation (the collected form of Appendix A's equations), with
# exp, log, sincos and each reciprocal counted as one operation.
F_RHS_Q = 60
# Bytes per ray of the shadow outputs copied back in the end-to-end timing:
# status 1, r/theta/phi/max|H| 4x8, steps 4, cell_i/cell_j 2x2, parity 1.
SHADOW_BYTES_PER_RAY = 42
DISK_BYTES_PER_RAY = 66  # + g, intensity, r_hit 3x8
ORACLE_SAMPLE_STRIDE = 128  # CPU baseline: every 128th pixel of each render
E2E_STEPS = 5  # end-to-end leg: steps timed with host copies (wall clock)
LOOSE_TOL = 1e-8  # the served stream's looser tolerance, where MIXED is meant to run
# DRAM bytes (read + write) of one FP64 trace launch over the 1024^2 set: ncu
# capture (one pass) of the timed launch of the current kernel, 47.60 MB read
# + 528.18 MB written (profiles/trace_fp64_persistent_kerr12x1024_dram.md);
# the outputs alone are 528.5 MB (42 B per ray).
FP64_TRAFFIC_BYTES_PER_LAUNCH = 575.78e6
# FP32-pipe (FMA heavy + lite) thread instructions, and warp instructions of
# every pipe, per double-float Cash-Karp attempt on the Kerr set: ncu capture
# of trace_df64_persistent on the 12 renders at 256x256 (3.3475e10 FMA-pipe
# warp instructions x 28.71 active lanes, and 4.050e10 warp instructions, over
# 2.7322e8 attempts), profiles/trace_df64_persistent_kerr12x256_ncu.md.
DF64_FP32_INST_PER_ATTEMPT = 3518
DF64_WARP_INST_PER_ATTEMPT = 148.2
# The same for the MIXED kernel (FP32 evaluations, FP32 stage sums) at tol
# 1e-8: ncu capture of trace_mixed_persistent on the 12 renders at 256x256
# (3.6500e9 FMA-pipe warp instructions x 25.19 active lanes, and 5.5962e9 warp
# instructions, over 1.4642e8 attempts),
# profiles/trace_mixed_persistent_kerr12x256_ncu.md.
MIXED_FP32_INST_PER_ATTEMPT = 628
MIXED_WARP_INST_PER_ATTEMPT = 38.22


def fp32_roofline(probe, inst_per_attempt, warp_inst_per_attempt, attempts, seconds):
    """Roofline of a kernel on the FP32 pipe (DF64, MIXED): its FMA-pipe thread
    instructions per attempt (ncu) x attempts/s over the FP32 probe's thread
    instruction rate, and, as `issue_frac`, its warp instructions of all pipes
    per attempt x attempts/s over the issue rate of one warp instruction per
    cycle per SM sub-partition, which the FP32 probe reaches."""
    rate = attempts * inst_per_attempt / seconds
    warp_peak = probe["fp32_fma"]["warp_inst_per_s"]
    return {"bound": "alu", "pipe": "FP32 (FMA heavy + lite)", "achieved": rate / 1e12,
            "peak": warp_peak * 32 / 1e12, "unit": "T thread-instructions/s",
            "frac": rate / (warp_peak * 32), "inst_per_attempt": inst_per_attempt,
            "issue_frac": attempts * warp_inst_per_attempt / seconds / warp_peak,
            "warp_inst_per_attempt": warp_inst_per_attempt,
            "peak_source": "FP32 pipe probe measured in this process"}


# Workloads: the headline Kerr set (default) and the measured "next" rows,
# each timed under the same rules. --side scales the pixel counts.
WORKLOADS = {
    "kerr": (WORKLOAD_NAME, METRIC),
    "qmetric": ("qmetric_shadow: 6 renders (q in {-0.5,0.1,0.5} x incl in {30,90} deg), "
                "r_obs=1000, SIDE^2 cell centres on [-8,8]^2, Cash-Karp tol 1e-10, "
                "r_cap=1.01*2, r_esc=1.1 r_obs, seeded 10-deg checkerboard",
                "rays/s (q-metric shadow renders, Cash-Karp)"),
    "disk_l0": ("paper_disk_figure: 3 constant-l0 thin-disk renders, (a, l0) in "
                "{(0,2.8),(0.5,2.8),(0.998,1.8)}, 85 deg, r_obs=1000, r_in=ISCO(a), r_out=20, "
                "2*SIDE x SIDE on [-24,24]x[-12,12], Cash-Karp tol 1e-10",
                "rays/s (constant-l0 disk renders, Cash-Karp)"),
    "uneven": ("uneven_batch: 256 requests from PCG64(4), side in {1,2,4,8}*SIDE/8, "
               "a~U[0,0.998], incl~U[5,85] deg, r_obs~U[500,2000], shadow [-8,8]^2 and "
               "disk (r_in=ISCO, r_out=20, [-25,25]^2) alternating, Cash-Karp tol 1e-10",
               "rays/s (uneven shadow/disk batch, Cash-Karp)"),
    "timelike": ("timelike: SIDE^2 unit-mass particles (E=1.2, L~U[-4,4], theta~U[0.3,pi-0.3], "
                 "p_theta=0, outward p_r from H=-1/2; PCG64 seed 7) from r=30 in Kerr a=0.9, "
                 "r_obs=1000, Cash-Karp tol 1e-10, explicit initial data",
                 "rays/s (time-like geodesics: unit-mass particles in Kerr, Cash-Karp)"),
}

TIMELIKE_A, TIMELIKE_R0, TIMELIKE_ROBS = 0.9, 30.0, 1000.0


def timelike_states(n, seed=7):
    """Initial data of the time-like workload: (states, E, L) with states rows
    (t, r, theta, phi, p_r, p_theta); p_r > 0 solves the mass shell
    g^tt E^2 - 2 g^tphi E L + g^phph L^2 + g^rr p_r^2 = -1 (Kerr, Boyer-Lindquist).
    Particles for which no real p_r exists are dropped."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a, r = TIMELIKE_A, TIMELIKE_R0
    th = rng.uniform(0.3, np.pi - 0.3, n)
    E = np.full(n, 1.2)
    L = rng.uniform(-4.0, 4.0, n)
    s2 = np.sin(th) ** 2
    sig = r * r + a * a * (1.0 - s2)
    dlt = r * r - 2.0 * r + a * a
    big_a = (r * r + a * a) ** 2 - a * a * dlt * s2
    gtt, gtp = -big_a / (sig * dlt), -2.0 * a * r / (sig * dlt)
    gpp, grr = (dlt - a * a * s2) / (sig * dlt * s2), dlt / sig
    rest = -1.0 - (gtt * E * E - 2.0 * gtp * E * L + gpp * L * L)
    keep = rest > 0.0
    st = np.zeros((int(keep.sum()), 6))
    st[:, 1] = r
    st[:, 2] = th[keep]
    st[:, 4] = np.sqrt(rest[keep] / grr[keep])
    return st, E[keep], L[keep]


def workload_renders(name, side):
    from paper_2202_00086_gb300 import workloads
    if name == "timelike":
        return []
    if name == "qmetric":
        return workloads.qmetric_shadow_set(side)
    if name == "disk_l0":
        return workloads.paper_disk_figure(2 * side, side)
    if name == "uneven":
        return workloads.uneven_batch(256, 4, sides=tuple(max(1, side * k // 8)
                                                            for k in (1, 2, 4, 8)))
    return workloads.kerr_shadow_ring_set(side)


def workload_label(name, side, tol=None):
    if name == "kerr":
        label = WORKLOAD_NAME.replace("1024x1024", "%dx%d" % (side, side))
    else:
        label = WORKLOADS[name][0].replace("SIDE", str(side))
    return label if tol is None else label.replace("tol 1e-10", "tol %g" % tol)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--workload", default="kerr", choices=sorted(WORKLOADS))
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="osiris", choices=["osiris", "reference"])
    p.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "df64"])
    p.add_argument("--kernel", default="batch", choices=["batch", "persistent", "plain"])
    p.add_argument("--side", type=int, default=1024)
    p.add_argument("--tol", type=float, default=None,
                   help="Cash-Karp tolerance of every render (default: the workload's, 1e-10)")
    p.add_argument("--block", type=int, default=0)
    p.add_argument("--rays-per-lane", type=int, default=0)
    p.add_argument("--refill-lanes", type=int, default=0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-variants", action="store_true")
    p.add_argument("--no-hbar", action="store_true")
    p.add_argument("--no-other-configs", action="store_true")
    p.add_argument("--hbar-side", type=int, default=512)
    p.add_argument("--serve-seconds", type=float, default=60.0)
    p.add_argument("--serve-rate", type=float, default=50.0)
    p.add_argument("--serve-baseline-seconds", type=float, default=5.0)
    p.add_argument("--serve-sustain-rate", default="auto",
                   help="second stream's arrival rate (renders/s): 'auto' = 10 above the "
                        "first stream's rate if the server kept up with it, else 85%% of "
                        "the capacity it measured; 0 = skip")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        return summarize_clock_lines(self.lines)


def summarize_clock_lines(lines):
    """The `clocks` object from nvidia-smi samples (ClockSampler.QUERY, csv,
    no header, no units): median and maximum SM clock, the throttle reasons
    seen Active in any sample, the sample count and the peak power."""
    sm, smax, reasons, power = [], [], set(), []
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            smax.append(float(f[2]))
            power.append(float(f[3]))
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
            "reasons": sorted(reasons), "samples": len(sm),
            "power_w_max": float(max(power))}


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ---------------------------------------------------------------------------

def oracle_sample_pixels(rd, stride):
    n = rd["nx"] * rd["ny"]
    return np.arange(stride // 2, n, stride, dtype=np.int64)


def oracle_options(oracle, rd):
    """The oracle's options for a render: disk radii and model, space-time."""
    opts = dict(tol=rd["tol"], cell_deg=rd["cell_deg"], cell_phase_deg=rd["cell_phase_deg"])
    if rd["mode"] == "disk":
        r_in = oracle.isco(rd["a"]) if rd["r_in"] == "isco" else rd["r_in"]
        opts.update(disk=True, r_in=r_in, r_out=rd["r_out"])
        if rd.get("l0") is not None:
            opts.update(disk_model=oracle.DISK_CONSTANT_L, l0=rd["l0"])
    if rd.get("q") is not None:
        opts.update(spacetime=oracle.QMETRIC, q=rd["q"])
    return opts


def run_oracle_sample(renders, stride):
    import oracle
    cores = os.cpu_count() or 1
    n = 0
    t0 = time.perf_counter()
    for rd in renders:
        pix = oracle_sample_pixels(rd, stride)
        oracle.trace_pixels(rd["a"], rd["r_obs"], rd["incl_deg"], rd["extent"], rd["nx"],
                            rd["ny"], pixels=pix, nthreads=cores, **oracle_options(oracle, rd))
        n += pix.size
    dt = time.perf_counter() - t0
    return n, dt, cores


def run_oracle_states(side, stride):
    """The time-like workload's oracle sample: every stride-th particle, one
    thread (the oracle's explicit-data entry is serial)."""
    import oracle
    st, E, L = timelike_states(side * side)
    sel = slice(stride // 2, None, stride)
    t0 = time.perf_counter()
    oracle.trace_states(TIMELIKE_A, TIMELIKE_ROBS, st[sel], E[sel], L[sel], mass2=1.0)
    return int(E[sel].size), time.perf_counter() - t0, 1


def oracle_leg(args, renders):
    """(rays, seconds, cores, description) of one pass of the oracle sample."""
    stride = ORACLE_SAMPLE_STRIDE
    if args.workload == "timelike":
        n, dt, cores = run_oracle_states(args.side, stride)
        return n, dt, cores, "every %dth particle (%d), one thread" % (stride, n)
    n, dt, cores = run_oracle_sample(renders, stride)
    return n, dt, cores, ("every %dth pixel of each of the %d renders (%d rays), all host cores"
                          % (stride, len(renders), n))


def reference_arm(args, renders):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        oracle_leg(args, renders)
    tot_n, tot_t, cores, sample = 0, 0.0, 1, ""
    for _ in range(args.steps):
        n, dt, cores, sample = oracle_leg(args, renders)
        tot_n += n
        tot_t += dt
    value = tot_n / tot_t
    sample += ", per step"
    line = {"impl": "reference", "metric": WORKLOADS[args.workload][1], "value": value,
            "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_label(args.workload, args.side, args.tol),
                       "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def measure_pipe_peaks(torch, osr, repeats=5):
    """Rates of the FP64 and FP32 pipes from the library's pipe probes: for
    each (precision, operation) the best of `repeats` launches that fill every
    SM, timed with CUDA events. Returns ({"fp64": FMA TFLOP/s, "fp32": FMA
    TFLOP/s}, details): the FMA rates are the flop peaks (2 operations per
    instruction), the multiply and add rates show the pipe's instruction rate
    for the other operations of the kernels."""
    iters = {osr.FP64: 2048, osr.MIXED: 32768}
    details = {}
    for prec, pname in ((osr.FP64, "fp64"), (osr.MIXED, "fp32")):
        for op, oname in ((osr.PROBE_FMA, "fma"), (osr.PROBE_MUL, "mul"), (osr.PROBE_ADD, "add")):
            n = osr.pipe_probe_threads(prec, op)
            out = torch.empty(n, dtype=torch.float64, device="cuda")
            osr.pipe_probe(prec, op, n, iters[prec], out)
            torch.cuda.synchronize()
            best = None
            for _ in range(repeats):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                fl = osr.pipe_probe(prec, op, n, iters[prec], out)
                e1.record()
                torch.cuda.synchronize()
                rate = fl / (e0.elapsed_time(e1) * 1e-3)
                best = rate if best is None or rate > best else best
            per_inst = 2.0 if op == osr.PROBE_FMA else 1.0
            details["%s_%s" % (pname, oname)] = {
                "tflops": best / 1e12, "warp_inst_per_s": best / per_inst / 32.0,
                "threads": n}
    peaks = {"fp64": details["fp64_fma"]["tflops"], "fp32": details["fp32_fma"]["tflops"]}
    return peaks, details


STREAM_LABEL = ("Poisson %g renders/s for %g s (PCG64 seed 5), side log-uniform 64..2048, "
                "a~U[0,0.998], incl~U[5,85] deg, r_obs=1000, shadow/disk 50/50, "
                "tol 1e-8/1e-10 50/50")


SERVED_FORM = ("DF64 for the renders at tol 1e-10, MIXED (FP32 stage evaluations and stage "
               "sums, df64 state) for those at tol 1e-8")


def serve_stream(osr, torch, dist, rank, world, barrier, rate, seconds, phase):
    """One served stream through the continuous-batching server in its served
    form (DF64, and MIXED for the renders at LOOSE_TOL; rounds as CUDA-graph
    launches of batch plans, each in-flight round on its own stream), renders
    dealt out whole to the GPUs. Returns the merged summary with latency
    windows."""
    from paper_2202_00086_gb300 import serve, workloads as wl
    all_arrivals = wl.served_stream(rate_hz=rate, duration_s=seconds)
    offered = sum(rd["nx"] * rd["ny"] for _, rd in all_arrivals)
    arrivals = serve.shard(all_arrivals, rank, world)
    barrier()
    srv = serve.RenderServer(precision=osr.DF64, loose_precision=osr.MIXED, loose_tol=LOOSE_TOL,
                             round_rays=1 << 21, cell_phase_deg=phase)
    summary = srv.run(arrivals, realtime=True)
    torch.cuda.synchronize()
    rec = serve.local_record(srv.done, srv.t0)
    recs = [rec]
    if dist is not None:
        recs = [None] * world
        dist.all_gather_object(recs, rec)
        summary = dict(serve.merge_records(recs, launches=summary["launches"]),
                       rejected=summary["rejected"])
    summary.update(serve.latency_windows(recs, seconds))
    summary["workload"] = STREAM_LABEL % (rate, seconds)
    summary["precision"] = SERVED_FORM
    summary["offered_rays_per_s"] = offered / seconds
    summary["mean_rays_per_render"] = offered / max(1, len(all_arrivals))
    # kept up: what had arrived by the last arrival was done within 2 s of it
    cap = max(summary["rays_per_s"] or 0.0, summary["offered_rays_per_s"])
    backlog = summary.get("backlog_rays_at_last_arrival")
    summary["kept_up"] = bool(backlog is not None and backlog <= 2.0 * cap)
    return summary


def serving_leg(args, osr, torch, dist, rank, world, barrier, phase):
    """The served-stream rows: the stream as specified (Poisson arrivals at
    --serve-rate for --serve-seconds) through continuous batching in the
    served form; a second stream that brackets the sustainable rate (with
    --serve-sustain-rate auto: 10 renders/s above the first stream's rate if
    the server kept up with it, else 85% of the capacity it measured, rounded
    down to 5 renders/s); and the one-render-per-launch FP64 baseline on the
    first --serve-baseline-seconds of the first stream. A stream is kept up
    with when the rays that had arrived by its last arrival were done within
    2 s of it."""
    from paper_2202_00086_gb300 import serve, workloads as wl
    main = serve_stream(osr, torch, dist, rank, world, barrier, args.serve_rate,
                        args.serve_seconds, phase)
    second = None
    if args.serve_sustain_rate != "0":
        if args.serve_sustain_rate == "auto":
            if main["kept_up"]:
                rate = args.serve_rate + 10.0
            else:
                cap = main["rays_per_s"] or 0.0
                rate = 5.0 * int(0.85 * cap / main["mean_rays_per_render"] / 5.0)
        else:
            rate = float(args.serve_sustain_rate)
        if rate > 0:
            second = serve_stream(osr, torch, dist, rank, world, barrier, rate,
                                  args.serve_seconds, phase)
            second["rate_renders_per_s"] = rate
    base_s = min(args.serve_baseline_seconds, args.serve_seconds)
    first = [x for x in wl.served_stream(rate_hz=args.serve_rate, duration_s=args.serve_seconds)
             if x[0] < base_s]
    mine = serve.shard(first, rank, world)
    barrier()
    base = serve.run_one_per_launch(mine, precision=osr.FP64, realtime=True,
                                    cell_phase_deg=phase)
    if dist is not None:
        brecs = [None] * world
        dist.all_gather_object(brecs, base["record"])
        base = serve.merge_records(brecs, launches=base["launches"])
    base.pop("record", None)
    base["workload"] = ("the first %g s of the same stream (%d renders), one plain FP64 "
                        "launch per render, each waited for" % (base_s, len(first)))
    return {"continuous_batching": main, "second_rate": second,
            "one_render_per_launch_fp64": base,
            "rays_per_s_ratio": (main["rays_per_s"] / base["rays_per_s"]
                                 if main["rays_per_s"] and base["rays_per_s"] else None)}


def other_configs(osr, torch, flush, stream, phase):
    """The target's other single-GPU configurations, each one launch timed
    with CUDA events after the L2 flush (a warm-up launch first, except for
    the 256-request batch, whose FP64 launch alone takes ~26 s), in FP64 and
    DF64: the 64^2 Schwarzschild shadow, the 2048^2 Schwarzschild thin disk
    (persistent grid) and the 256 uneven requests of PCG64(4) in one batched
    launch."""
    from paper_2202_00086_gb300 import workloads as wl

    def timed(fn, warm=True):
        if warm:
            fn()
            torch.cuda.synchronize()
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e-3

    res = {}
    ws = torch.empty(osr.workspace_bytes(256), dtype=torch.uint8, device="cuda")
    for key, rd in (("config1_schwarzschild_shadow_64x64", wl.schwarzschild_shadow_64()),
                    ("config3_schwarzschild_disk_2048x2048", wl.schwarzschild_disk())):
        cam = osr.Camera.from_render(rd)
        disk = rd["mode"] == "disk"
        out = osr.alloc_outputs(cam.n_rays, fields=osr.DISK_FIELDS if disk else osr.SHADOW_FIELDS)
        row = {"rays": cam.n_rays}
        for prec, pn in ((osr.FP64, "fp64"), (osr.DF64, "df64")):
            kw = dict(out=out, tol=rd["tol"], precision=prec, persistent=True, workspace=ws,
                      cell_phase_deg=rd["cell_phase_deg"])
            if disk:
                t = timed(lambda: osr.render_disk(cam, rd["r_in"], rd["r_out"], **kw))
            else:
                t = timed(lambda: osr.trace(cam, **kw))
            row[pn + "_rays_per_s"] = cam.n_rays / t
        res[key] = row
    rds = wl.uneven_batch()
    cams = [osr.Camera.from_render(rd) for rd in rds]
    outs = [osr.alloc_outputs(c.n_rays, fields=osr.DISK_FIELDS if rd["mode"] == "disk"
                              else osr.SHADOW_FIELDS) for c, rd in zip(cams, rds)]
    reqs = [{"camera": c, "out": o, "tol": rd["tol"], "disk": rd["mode"] == "disk",
             "r_in": osr.resolve_r_in(rd) if rd["mode"] == "disk" else 0.0,
             "r_out": rd["r_out"] if rd["mode"] == "disk" else 0.0}
            for c, o, rd in zip(cams, outs, rds)]
    n = sum(c.n_rays for c in cams)
    row = {"rays": n, "requests": len(rds)}
    for prec, pn in ((osr.FP64, "fp64"), (osr.DF64, "df64")):
        t = timed(lambda: osr.trace_batch(reqs, workspace=ws, precision=prec,
                                          cell_phase_deg=phase), warm=False)
        row[pn + "_rays_per_s"] = n / t
    res["config4_uneven_256_requests_sides_128_to_1024"] = row
    return res


def h_distribution(status, max_abs_H, bar=1e-10):
    """Per-status distribution of the per-ray max |H| (Sec. 3.1, Error =
    |H_num|): count, p50, p99, max and the share of rays below `bar`."""
    out = {}
    for name, code in (("captured", 1), ("escaped", 2), ("disk", 3)):
        h = max_abs_H[status == code]
        if h.size == 0:
            continue
        out[name] = {"n": int(h.size), "p50": float(np.percentile(h, 50)),
                     "p99": float(np.percentile(h, 99)), "max": float(h.max()),
                     "frac_below_bar": float((h < bar).mean())}
    return out


H_BAR = 1e-10  # the |H| bar of the target (Sec. 3.1 reports the error as |H_num|)


def h_of_outputs(renders, outs, normalised=True):
    """Per-status max-|H| distribution over every ray of the renders' device
    outputs, and (captured rays) the normalised |H| of captured_h_normalised."""
    st = np.concatenate([o["status"].cpu().numpy() for o in outs])
    hh = np.concatenate([o["max_abs_H"].cpu().numpy() for o in outs])
    res = {"by_status": h_distribution(st, hh, H_BAR)}
    if normalised:
        parts = [captured_h_normalised(rd, o["status"].cpu().numpy(), o["r"].cpu().numpy(),
                                       o["theta"].cpu().numpy(), o["max_abs_H"].cpu().numpy())
                 for rd, o in zip(renders, outs)]
        v = np.concatenate([x for x in parts if x is not None])
        if v.size:
            res["captured_normalised"] = {"p50": float(np.percentile(v, 50)),
                                          "p99": float(np.percentile(v, 99)),
                                          "max": float(v.max())}
    return res


def first_tol_meeting(points, bar=H_BAR):
    """Per integrator, the loosest swept tolerance at which every escaped ray,
    every captured ray, and every ray keeps max |H| below the bar (None when
    no swept tolerance does)."""
    out = {}
    for iname in sorted({p["integrator"] for p in points}):
        rows = sorted((p for p in points if p["integrator"] == iname), key=lambda p: -p["tol"])
        res = {}
        for cls in ("escaped", "captured", "all"):
            res[cls] = None
            for p in rows:
                bs = p["by_status"]
                mx = (max(v["max"] for v in bs.values()) if cls == "all"
                      else bs.get(cls, {"max": 0.0})["max"])
                if mx < bar:
                    res[cls] = {"tol": p["tol"], "rays_per_s": p["rays_per_s"]}
                    break
        out[iname] = res
    return out


def captured_h_normalised(rd, status, r, theta, max_abs_H):
    """max |H| of captured rays relative to the size of the terms of 2H at the
    capture point. With H = N / (2 Sigma), N = Delta p_r^2 + p_theta^2 + W^2
    - P^2 / Delta and P = (r^2 + a^2) E - a L, the positive terms sum to
    P^2 / Delta on the constraint surface, so the terms of 2H sum to
    2 P^2 / (Delta Sigma) and |2H| / sum|terms| = |H| Delta Sigma / P^2.
    E and L of each pixel are those of the zero-angular-momentum observer
    of Sec. 2.3 (Kerr metric at the observer)."""
    cap = status == 1
    if not cap.any():
        return None
    a, r0, th0 = rd["a"], rd["r_obs"], np.radians(rd["incl_deg"])
    x0, x1, y0, y1 = rd["extent"]
    nx, ny = rd["nx"], rd["ny"]
    idx = np.flatnonzero(cap)
    x = x0 + (idx % nx + 0.5) * (x1 - x0) / nx
    s2, c2 = np.sin(th0) ** 2, np.cos(th0) ** 2
    sig0, dlt0 = r0 * r0 + a * a * c2, r0 * r0 - 2 * r0 + a * a
    g_tph = -2 * a * r0 * s2 / sig0
    g_pp = s2 * ((r0 * r0 + a * a) ** 2 - a * a * dlt0 * s2) / sig0
    E = np.sqrt(dlt0 * s2 / g_pp) + x * g_tph / (r0 * np.sqrt(g_pp))
    L = -x * np.sqrt(g_pp) / r0
    rr, cc = r[idx], np.cos(theta[idx])
    sig = rr * rr + a * a * cc * cc
    dlt = rr * rr - 2 * rr + a * a
    P = (rr * rr + a * a) * E - a * L
    return max_abs_H[idx] * dlt * sig / (P * P)


def main():
    args = parse()
    renders = workload_renders(args.workload, args.side)
    if args.tol is not None:
        renders = [dict(rd, tol=args.tol) for rd in renders]
    if args.impl == "reference":
        return reference_arm(args, renders)

    import torch
    import paper_2202_00086_gb300 as osr

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    precision = {"fp64": osr.FP64, "mixed": osr.MIXED, "df64": osr.DF64}[args.precision]
    tol = 1e-10 if args.tol is None else args.tol
    f_rhs = F_RHS_Q if args.workload == "qmetric" else F_RHS
    timelike = args.workload == "timelike"
    cams = [osr.Camera.from_render(rd) for rd in renders]
    disk = [rd["mode"] == "disk" for rd in renders]
    if timelike:
        st_np, e_np, l_np = timelike_states(args.side * args.side)
        tl = [torch.tensor(x, device="cuda").contiguous() for x in (st_np, e_np, l_np)]
        sizes = [int(e_np.size)]
        outs = [osr.alloc_outputs(sizes[0])]
    else:
        sizes = [c.n_rays for c in cams]
        outs = [osr.alloc_outputs(c.n_rays, fields=osr.DISK_FIELDS if d else osr.SHADOW_FIELDS)
                for c, d in zip(cams, disk)]
    n_rays = sum(sizes)
    ws = torch.empty(osr.workspace_bytes(max(1, len(cams))), dtype=torch.uint8, device="cuda")
    stats = osr.new_stats()
    stream = torch.cuda.current_stream()
    launches = [0]
    from paper_2202_00086_gb300 import workloads
    cell_deg = renders[0]["cell_deg"] if renders else 10.0
    cell_phase = renders[0]["cell_phase_deg"] if renders else workloads.checker_phase_deg(2202)
    common = dict(tol=tol, precision=precision, block_size=args.block, workspace=ws,
                  cell_deg=cell_deg, cell_phase_deg=cell_phase,
                  rays_per_lane=args.rays_per_lane, refill_lanes=args.refill_lanes)

    def request(rd, c, o):
        r = {"camera": c, "out": o, "tol": rd["tol"]}
        if rd["mode"] == "disk":
            r.update(disk=True, r_in=osr.resolve_r_in(rd), r_out=rd["r_out"], l0=rd.get("l0"))
        return r

    reqs = [request(rd, c, o) for rd, c, o in zip(renders, cams, outs)]

    def trace_one(rd, c, o, **kw):
        if rd["mode"] == "disk":
            osr.render_disk(c, osr.resolve_r_in(rd), rd["r_out"], out=o, l0=rd.get("l0"), **kw)
        else:
            osr.trace(c, out=o, **kw)

    def launch_all(st, opts):
        if timelike:
            osr.trace_states(TIMELIKE_A, TIMELIKE_ROBS, tl[0], tl[1], tl[2], out=outs[0],
                             mass2=1.0, persistent=True, stats=st, **opts)
            launches[0] += 1
        elif args.kernel == "batch":
            osr.trace_batch(reqs, stats=st, **opts)
            launches[0] += 1
        else:
            for rd, c, o in zip(renders, cams, outs):
                trace_one(rd, c, o, persistent=(args.kernel == "persistent"), stats=st, **opts)
                launches[0] += 1

    def step(st=None):
        launch_all(st, common)

    # L2 flush buffer (larger than the 129 MB L2), written between timed steps
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # Pipe probes (roofline denominators), same process: 16 independent chains
    # per thread of one operation, every SM filled with resident blocks
    peaks, probe = measure_pipe_peaks(torch, osr)

    # ---- timed region: K steps, per-step CUDA events, L2 flushed between ----
    clocks = ClockSampler(local)
    stats.zero_()
    launches[0] = 0
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        ev[k][0].record(stream)
        step(stats)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    barrier()
    clk = clocks.stop()
    kernel_launches = launches[0]
    ms = sum(a.elapsed_time(b) for a, b in ev)
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    s = osr.decode_stats(stats)

    # per-status max |H| of the last timed step (the headline launch itself)
    hbar = None
    if not args.no_hbar and args.workload == "kerr" and precision == osr.FP64:
        hbar = {"bar": H_BAR, "ck45_tol1e-10": h_of_outputs(renders, outs)}

    # ---- end to end through the C interface with host buffers ----
    e2e = None
    if not args.no_e2e:
        host = [osr.alloc_outputs(n, device="cpu", pin_memory=True,
                                  fields=osr.DISK_FIELDS if d else osr.SHADOW_FIELDS)
                for n, d in zip(sizes, disk if not timelike else [False])]
        h2d = osr.workspace_bytes(len(cams)) - 256 if args.kernel == "batch" else 0
        d2h = sum((DISK_BYTES_PER_RAY if d else SHADOW_BYTES_PER_RAY) * n
                  for n, d in zip(sizes, disk if not timelike else [False]))
        e2e_step, e2e_api = step, "per-render calls"
        if timelike:
            # the particles' initial data come from pinned host memory every step
            tl_host = [torch.from_numpy(x).contiguous().pin_memory() for x in (st_np, e_np, l_np)]
            h2d = sum(x.numel() * x.element_size() for x in tl_host)

            def e2e_states():
                for dst, src in zip(tl, tl_host):
                    dst.copy_(src, non_blocking=True)
                step()
            e2e_step, e2e_api = e2e_states, "osiris_trace_states_ex"
        elif args.kernel == "batch":
            # the serving API: a batch plan uploads the request table from its
            # pinned staging table and launches one CUDA graph per step
            ws_plan = torch.empty(osr.workspace_bytes(len(cams)), dtype=torch.uint8,
                                  device="cuda")
            plan = osr.BatchPlan(len(cams), spacetime=(osr.SPACETIME_QMETRIC
                                                       if args.workload == "qmetric"
                                                       else osr.SPACETIME_KERR),
                                 **dict(common, workspace=ws_plan))
            e2e_step, e2e_api = (lambda: plan.launch(reqs)), "osiris_batch_plan_launch"
            e2e_step()  # first launch outside the timed region, like the warm-up steps
        # the same step as the device-timed region, at most E2E_STEPS of them
        e2e_steps = max(1, min(args.steps, E2E_STEPS))
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(e2e_steps):
            e2e_step()
            for n, o, h in zip(sizes, outs, host):
                osr.copy_outputs_to_host(o, h, n)
            torch.cuda.synchronize()
        te = time.perf_counter() - t0
        tt = torch.tensor([te], dtype=torch.float64, device="cuda")
        if dist is not None:
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        te = float(tt.item())
        e2e = {"value": world * n_rays * e2e_steps / te, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "api": e2e_api,
               "steps": e2e_steps}

    def timed_variant(vstep):
        """Warm-up, then args.steps device-timed calls of vstep(stats) with
        the L2 flushed between them; returns (ms over all steps, max over
        ranks; decoded stats)."""
        vstats = osr.new_stats()
        for _ in range(max(1, args.warmup)):
            vstep(None)
        torch.cuda.synchronize()
        vev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        barrier()
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(k & 0xff)
            vev[k][0].record(stream)
            vstep(vstats)
            vev[k][1].record(stream)
        torch.cuda.synchronize()
        barrier()
        vms = sum(a.elapsed_time(b) for a, b in vev)
        tv = torch.tensor([vms], dtype=torch.float64, device="cuda")
        if dist is not None:
            dist.all_reduce(tv, op=dist.ReduceOp.MAX)
        return float(tv.item()), osr.decode_stats(vstats)

    # ---- double-float variant on the same workload (same rules, own timing) ----
    variants = {}
    if precision == osr.FP64 and not args.no_variants:
        vcommon = dict(common, precision=osr.DF64)
        vms, vs = timed_variant(lambda st: launch_all(st, vcommon))
        vatt = vs["accepted"] + vs["rejected"] + vs["root_steps"]
        vflops = vs["rhs_evals"] * f_rhs + vatt * F_STEP
        variants["df64"] = {
            "value": world * n_rays * args.steps / (vms * 1e-3), "unit": UNIT,
            "ms_per_step": vms / args.steps,
            "rhs_evals_per_s": world * vs["rhs_evals"] / (vms * 1e-3),
            "speedup_vs_fp64": ms_max / vms,
            "dtype": "f64+df64",
            "fp64_equivalent_tflops": vflops / (vms * 1e-3) / 1e12,
            "fp64_equivalent_frac_of_fp64_peak": vflops / (vms * 1e-3) / 1e12 / peaks["fp64"],
            # the pipe the double-float kernel runs on (see fp32_roofline)
            "roofline": (fp32_roofline(probe, DF64_FP32_INST_PER_ATTEMPT,
                                       DF64_WARP_INST_PER_ATTEMPT, vatt, vms * 1e-3)
                if args.workload == "kerr" else None),
            "max_abs_H": vs["max_abs_H"],
            "steps_per_ray": {"accepted": vs["accepted"] / (n_rays * args.steps),
                              "rejected": vs["rejected"] / (n_rays * args.steps),
                              "locate": vs["root_steps"] / (n_rays * args.steps)},
        }

    # ---- the three precisions at the looser tolerance MIXED is meant for ----
    if (precision == osr.FP64 and not args.no_variants and args.workload in ("kerr", "qmetric")
            and args.kernel == "batch"):
        reqs_loose = [dict(r, tol=LOOSE_TOL) for r in reqs]
        loose = {"workload": "the same renders at Cash-Karp tol %g" % LOOSE_TOL}
        for name, prec in (("fp64", osr.FP64), ("df64", osr.DF64), ("mixed", osr.MIXED)):
            lopts = dict(common, precision=prec)
            lms, ls = timed_variant(lambda st, o=lopts: osr.trace_batch(reqs_loose, stats=st, **o))
            loose[name] = {"value": world * n_rays * args.steps / (lms * 1e-3), "unit": UNIT,
                           "ms_per_step": lms / args.steps,
                           "accepted_per_ray": ls["accepted"] / (n_rays * args.steps),
                           "rejected_per_ray": ls["rejected"] / (n_rays * args.steps)}
            if prec in (osr.DF64, osr.MIXED) and args.workload == "kerr":
                # against the FP32 pipe DF64 and MIXED run on, as variants.df64
                mixed = prec == osr.MIXED
                loose[name]["roofline"] = fp32_roofline(
                    probe, MIXED_FP32_INST_PER_ATTEMPT if mixed else DF64_FP32_INST_PER_ATTEMPT,
                    MIXED_WARP_INST_PER_ATTEMPT if mixed else DF64_WARP_INST_PER_ATTEMPT,
                    ls["accepted"] + ls["rejected"] + ls["root_steps"], lms * 1e-3)
        loose["mixed_vs_df64"] = loose["mixed"]["value"] / loose["df64"]["value"]
        variants["tol_%g" % LOOSE_TOL] = loose

    # ---- the |H| bar: Dormand-Prince on the same launch, and a tolerance sweep ----
    if hbar is not None:
        def one_launch(rds, integrator, tol_):
            cs = [osr.Camera.from_render(rd) for rd in rds]
            os_ = [osr.alloc_outputs(c.n_rays) for c in cs]
            w = torch.empty(osr.workspace_bytes(len(cs)), dtype=torch.uint8, device="cuda")
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            osr.trace_batch([{"camera": c, "out": o} for c, o in zip(cs, os_)], workspace=w,
                            tol=tol_, integrator=integrator, cell_deg=cell_deg,
                            cell_phase_deg=cell_phase)
            e1.record(stream)
            torch.cuda.synchronize()
            return os_, sum(c.n_rays for c in cs) / (e0.elapsed_time(e1) * 1e-3)

        dp_outs, dp_rate = one_launch(renders, osr.RKDP45, tol)
        hbar["dp45_tol1e-10"] = h_of_outputs(renders, dp_outs)
        hbar["dp45_tol1e-10"]["rays_per_s"] = dp_rate
        del dp_outs
        side = args.hbar_side
        small = workloads.kerr_shadow_ring_set(side)
        sweep = []
        for integ, iname in ((osr.RKCK45, "ck45"), (osr.RKDP45, "dp45")):
            for tol_ in (1e-10, 1e-11, 1e-12):
                o_, rate = one_launch(small, integ, tol_)
                row = h_of_outputs(small, o_, normalised=False)
                sweep.append({"integrator": iname, "tol": tol_, "rays_per_s": rate,
                              "by_status": row["by_status"]})
        hbar["sweep"] = {"renders": "the same 12 renders at %dx%d" % (side, side),
                         "points": sweep, "first_tol_meeting_bar": first_tol_meeting(sweep)}

    # ---- the other single-GPU configurations (one timed launch each) ----
    configs = None
    if (not args.no_other_configs and args.workload == "kerr" and precision == osr.FP64
            and args.side == 1024):
        configs = other_configs(osr, torch, flush, stream, cell_phase)

    # ---- served render stream: continuous batching (DF64 + MIXED) vs one
    # render per launch (FP64 plain kernel), the same Poisson arrivals ----
    serving = None
    if args.serve_seconds > 0 and precision == osr.FP64 and args.workload == "kerr":
        serving = serving_leg(args, osr, torch, dist, rank, world, barrier,
                              common["cell_phase_deg"])

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n, dt, cores, sample = oracle_leg(args, renders)
        cpu = {"value": n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": sample + ", one pass"}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    value = world * n_rays * args.steps / (ms_max * 1e-3)
    attempts = s["accepted"] + s["rejected"] + s["root_steps"]
    flops = s["rhs_evals"] * f_rhs + attempts * F_STEP
    per_launch_ms = ms / max(1, kernel_launches)
    achieved = flops / max(1, kernel_launches) / (per_launch_ms * 1e-3) / 1e12
    peak = peaks["fp64"] if precision == osr.FP64 else peaks["fp32"]
    # The headline roofline: FP64 operations against the FP64 pipe for the FP64
    # kernels; for DF64 and MIXED, the FP32 pipe and the issue slots they run
    # on, from instruction counts measured on the Kerr set (else none).
    if precision == osr.FP64:
        roofline_main = {
            "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak,
            "traffic": (FP64_TRAFFIC_BYTES_PER_LAUNCH
                        if args.side == 1024 and args.kernel == "batch"
                        and args.workload == "kerr" else None),
            "peak_source": ("pipe probe measured in this process: FP64 fused "
                            "multiply-add, 16 chains per thread, every SM full"),
            "flops_per_launch": flops / max(1, kernel_launches),
            "f_rhs": f_rhs, "f_step": F_STEP}
    elif args.workload == "kerr":
        mixed = precision == osr.MIXED
        roofline_main = fp32_roofline(
            probe, MIXED_FP32_INST_PER_ATTEMPT if mixed else DF64_FP32_INST_PER_ATTEMPT,
            MIXED_WARP_INST_PER_ATTEMPT if mixed else DF64_WARP_INST_PER_ATTEMPT,
            attempts / max(1, kernel_launches), per_launch_ms * 1e-3)
    else:
        roofline_main = None
    line = {
        "metric": WORKLOADS[args.workload][1], "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {osr.FP64: "f64", osr.MIXED: "f64+f32", osr.DF64: "f64+df64"}[precision],
        "data": "synthetic",
        "config": {"workload": workload_label(args.workload, args.side, args.tol),
                   "rays_per_step_per_gpu": n_rays,
                   "kernel": args.kernel, "precision": args.precision,
                   "l2": "flushed between timed steps (256 MB write)",
                   "wall_s_timed": t_wall},
        "rhs_evals_per_s": world * s["rhs_evals"] / (ms_max * 1e-3),
        "steps_per_ray": {"accepted": s["accepted"] / (n_rays * args.steps),
                          "rejected": s["rejected"] / (n_rays * args.steps),
                          "locate": s["root_steps"] / (n_rays * args.steps)},
        "status_counts_per_step": {k: s[k] // args.steps for k in
                                   ("status_captured", "status_escaped", "status_maxstep",
                                    "status_disk", "status_error")},
        "max_abs_H": s["max_abs_H"],
        "roofline": roofline_main,
        "fma_probe_tflops": peaks,
        "pipe_probes": probe,
        "variants": variants,
        "serving": serving,
        "hbar": hbar,
        "other_configs": configs,
        "clocks": clk,
        "gpu_launches": kernel_launches,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
