"""Launch autotuner for the persistent trace kernels.

Times candidate launches of a precision / integrator pair on a sample render
set (one batched persistent launch each), keeps the fastest and caches it
per GPU model in a JSON file. `tuned_opts` returns the cached choice as
keyword arguments for the trace calls. The search has two stages:
  1. launch shape: threads per block x resident blocks per SM (0 = the
     occupancy limit), with the library's default work distribution;
  2. work granularity at the best shape: rays per lane (a lane claims that
     many consecutive rays from the device queue with each warp atomic) x
     refill granularity (a warp whose other lanes are still integrating
     refills its idle lanes only once at least that many are idle).
Rays are independent, so every candidate gives the same outputs; only the
time differs.
"""
import json
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(_HERE, "_build", "autotune.json")
BLOCKS = (64, 96, 128, 192, 256)
PER_SM = (0, 1, 2, 3, 4)  # 0 = the occupancy limit
RAYS_PER_LANE = (1, 2, 4)
REFILL_LANES = (1, 2, 4, 8, 16, 32)
DEFAULT_GRANULARITY = (0, 0)  # the library's default (one ray per lane; refill at 4 idle
#                               lanes, 32 in MIXED)
KEYS = ("block_size", "blocks_per_sm", "rays_per_lane", "refill_lanes")


def candidates(blocks=BLOCKS, per_sm=PER_SM):
    """Launch shapes of the first stage: (block, blocks per SM)."""
    return [(b, k) for b in blocks for k in per_sm]


def granularity_candidates(rays=RAYS_PER_LANE, refill=REFILL_LANES):
    """Work granularities of the second stage: (rays per lane, refill lanes)."""
    return [(r, f) for r in rays for f in refill]


def choose(timings):
    """Fastest candidate from {candidate tuple: seconds}; ties go to the
    smaller tuple (smaller block, the occupancy-limited grid, the library's
    default work distribution)."""
    if not timings:
        raise ValueError("no candidate ran")
    return min(timings, key=lambda c: (timings[c], c))


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


def autotune(precision=None, integrator=0, renders=None, cands=None, grans=None, repeats=2,
             cache_path=DEFAULT_CACHE, timer=None):
    """Time each launch shape of `cands` (stage 1), then each work
    granularity of `grans` at the fastest shape (stage 2), on `renders`
    (default: the 12-render Kerr set at 256x256) in one batched persistent
    launch per timing. Returns (best, timings): best = (block, blocks per
    SM, rays per lane, refill lanes), timings keyed by such 4-tuples. The
    best candidate, its time and the spread of all timings go to the cache.
    `timer(block, per_sm, rays_per_lane, refill_lanes)` may replace the GPU
    timing (tests)."""
    import paper_2202_00086_gb300 as osr
    precision = osr.DF64 if precision is None else precision
    cands = candidates() if cands is None else cands
    grans = granularity_candidates() if grans is None else grans
    if timer is None:
        timer, device = _gpu_timer(osr, precision, integrator, renders, repeats)
    else:
        device = "test-device"
    timings = {}

    def run(c):
        try:
            timings[c] = timer(*c)
        except osr.OsirisError:
            pass  # e.g. more blocks per SM than the registers allow

    for b, k in cands:
        run((b, k) + DEFAULT_GRANULARITY)
    b, k, _, _ = choose(timings)
    for r, f in grans:
        if (b, k, r, f) not in timings:
            run((b, k, r, f))
    best = choose({c: t for c, t in timings.items() if c[:2] == (b, k)})
    cache = load_cache(cache_path)
    entry = dict(zip(KEYS, best))
    entry.update(seconds=timings[best], slowest_seconds=max(timings.values()),
                 candidates=len(timings))
    cache[_key(device, precision, integrator)] = entry
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
    return {k: entry[k] for k in KEYS if k in entry}


def _gpu_timer(osr, precision, integrator, renders, repeats):
    import torch
    from . import workloads
    if renders is None:
        renders = workloads.kerr_shadow_ring_set(256)
    cams = [osr.Camera.from_render(rd) for rd in renders]
    outs = [osr.alloc_outputs(c.n_rays) for c in cams]
    ws = torch.empty(osr.workspace_bytes(len(cams)), dtype=torch.uint8, device="cuda")
    reqs = [{"camera": c, "out": o, "tol": rd["tol"]} for c, o, rd in zip(cams, outs, renders)]

    def timer(block, per_sm, rays_per_lane=0, refill_lanes=0):
        best = float("inf")
        for _ in range(repeats):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            osr.trace_batch(reqs, workspace=ws, precision=precision, integrator=integrator,
                            block_size=block, blocks_per_sm=per_sm, rays_per_lane=rays_per_lane,
                            refill_lanes=refill_lanes)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) * 1e-3)
        return best

    return timer, torch.cuda.get_device_name()
