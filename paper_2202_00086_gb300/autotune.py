"""Launch-shape autotuner for the persistent trace kernels.

Times every candidate (threads per block x resident blocks per SM) of a
precision / integrator pair on a sample render set, keeps the fastest and
caches it per GPU model in a JSON file. `tuned_opts` returns the cached
choice as keyword arguments for the trace calls.

Two launch parameters are fixed by the kernel design rather than tuned:
  - rays per thread = 1: a lane's whole ray state lives in registers, and the
    register budget (FP64: ~200, DF64: 128 per thread) leaves no room for a
    second ray;
  - refill granularity = 1 warp-wide atomic as soon as any lane is idle: a
    ray start costs about one evaluation of the equations against ~350
    attempts per ray, so waiting for more idle lanes would only add idle
    lane-cycles.
"""
import json
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(_HERE, "_build", "autotune.json")
BLOCKS = (64, 96, 128, 192, 256)
PER_SM = (0, 1, 2, 3, 4)  # 0 = the occupancy limit


def candidates(blocks=BLOCKS, per_sm=PER_SM):
    return [(b, k) for b in blocks for k in per_sm]


def choose(timings):
    """Fastest candidate from {(block, per_sm): seconds}; ties go to the
    smaller block, then to the occupancy-limited grid (per_sm = 0)."""
    if not timings:
        raise ValueError("no candidate ran")
    return min(timings, key=lambda c: (timings[c], c[0], c[1]))


def _key(device_name, precision, integrator):
    return "%s|precision=%d|integrator=%d" % (device_name, precision, integrator)


def load_cache(path=DEFAULT_CACHE):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache, path=DEFAULT_CACHE):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def autotune(precision=None, integrator=0, renders=None, cands=None, repeats=2,
             cache_path=DEFAULT_CACHE, timer=None):
    """Time each candidate on `renders` (default: the 12-render Kerr set at
    256x256) in one batched persistent launch; return (best, timings) and
    store best in the cache. `timer(block, per_sm)` may replace the GPU
    timing (tests)."""
    import paper_2202_00086_gb300 as osr
    precision = osr.DF64 if precision is None else precision
    cands = candidates() if cands is None else cands
    if timer is None:
        timer, device = _gpu_timer(osr, precision, integrator, renders, repeats)
    else:
        device = "test-device"
    timings = {}
    for b, k in cands:
        try:
            timings[(b, k)] = timer(b, k)
        except osr.OsirisError:
            continue  # e.g. more blocks per SM than the registers allow
    best = choose(timings)
    cache = load_cache(cache_path)
    cache[_key(device, precision, integrator)] = {"block_size": best[0], "blocks_per_sm": best[1],
                                                 "seconds": timings[best]}
    save_cache(cache, cache_path)
    return best, timings


def tuned_opts(precision, integrator=0, cache_path=DEFAULT_CACHE, device_name=None):
    """Cached launch shape as trace keyword arguments ({} when not tuned)."""
    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_name()
    entry = load_cache(cache_path).get(_key(device_name, precision, integrator))
    if not entry:
        return {}
    return {"block_size": entry["block_size"], "blocks_per_sm": entry["blocks_per_sm"]}


def _gpu_timer(osr, precision, integrator, renders, repeats):
    import torch
    from . import workloads
    if renders is None:
        renders = workloads.kerr_shadow_ring_set(256)
    cams = [osr.Camera.from_render(rd) for rd in renders]
    outs = [osr.alloc_outputs(c.n_rays) for c in cams]
    ws = torch.empty(osr.workspace_bytes(len(cams)), dtype=torch.uint8, device="cuda")
    reqs = [{"camera": c, "out": o, "tol": rd["tol"]} for c, o, rd in zip(cams, outs, renders)]

    def timer(block, per_sm):
        best = float("inf")
        for _ in range(repeats):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            osr.trace_batch(reqs, workspace=ws, precision=precision, integrator=integrator,
                            block_size=block, blocks_per_sm=per_sm)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) * 1e-3)
        return best

    return timer, torch.cuda.get_device_name()
