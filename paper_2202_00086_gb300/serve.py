"""Continuous-batching render server.

Renders (camera set-ups) arrive over time. The server:
  - admits a waiting render when its output buffers fit in an HBM budget
    (outputs stay on the device until the render completes);
  - runs rounds: each round is ONE persistent batched launch over pixel
    ranges of every active render, so renders that arrive while others are on
    the GPU join the next round and their rays share launches with the older
    renders'. With graphs (the default) each in-flight slot owns a batch plan
    (osiris_batch_plan_*): table upload, queue reset and kernel recorded once
    as a CUDA graph, so a round is one graph launch with patched arguments;
    without, a round is one osiris_trace_batch call;
  - keeps up to `max_inflight` rounds queued on the stream, so the GPU never
    waits for the host between rounds;
  - detects round completion with CUDA events and timestamps each render at
    the completion of its last pixel range.

Round composition: a batched launch holds one space-time and one precision,
so each render has a kind: Kerr renders run at the server's precision, and
q-metric renders (shadow and lensing; Appendix A) too, except that a MIXED
server runs them in FP64 (the q-metric has no MIXED kernel). A round serves one
kind: that of the oldest render with rays left, or the next kind in that
order when the previous round served it, so kinds alternate while several
have work. Within the round every active render of the kind first receives up
to `min_chunk` rays in arrival order (small renders finish in one round),
then the rest of the round budget goes to the oldest of them. Rays are independent, so a
render's outputs are the same whether it runs alone or in a mix (the GPU
tests check this bitwise).

The scheduler is host code; every ray is traced by the CUDA kernels of the
library. For tests without a GPU the launch, allocation and event functions
can be replaced.
"""
import collections
import time

import numpy as np

SHADOW_BYTES_PER_RAY = 42  # status 1, r/theta/phi/max|H| 32, steps 4, cells 4, parity 1
DISK_BYTES_PER_RAY = 66    # + g, intensity, r_hit


class ServedRender:
    __slots__ = ("rid", "render", "arrival", "camera", "disk", "r_in", "r_out", "tol",
                 "n_rays", "next_ray", "rays_done", "out", "bytes", "t_submit", "t_admit",
                 "t_done", "chunks", "kind")

    def __init__(self, rid, render, arrival):
        self.rid = rid
        self.render = render
        self.arrival = arrival
        self.disk = render["mode"] == "disk"
        self.n_rays = render["nx"] * render["ny"]
        self.bytes = self.n_rays * (DISK_BYTES_PER_RAY if self.disk else SHADOW_BYTES_PER_RAY)
        self.next_ray = 0
        self.rays_done = 0
        self.camera = None
        self.out = None
        self.r_in = self.r_out = 0.0
        self.tol = render["tol"]
        self.t_submit = self.t_admit = self.t_done = None
        self.chunks = []  # (first_ray, n_rays) in launch order
        self.kind = None  # (space-time, precision) of the launches that trace it


class _Round:
    __slots__ = ("event", "parts", "ws_index", "t_launch")

    def __init__(self, event, parts, ws_index, t_launch):
        self.event = event
        self.parts = parts
        self.ws_index = ws_index
        self.t_launch = t_launch


class RenderServer:
    def __init__(self, precision=None, round_rays=1 << 21, min_chunk=1 << 14,
                 hbm_budget_bytes=8 << 30, max_inflight=2, max_entries=4096,
                 keep_outputs=False, cell_deg=10.0, cell_phase_deg=0.0, backend=None,
                 clock=time.perf_counter, graphs=True):
        import paper_2202_00086_gb300 as osr
        self.osr = osr
        self.precision = osr.DF64 if precision is None else precision
        self.round_rays = int(round_rays)
        self.min_chunk = int(min_chunk)
        self.hbm_budget = int(hbm_budget_bytes)
        self.max_inflight = int(max_inflight)
        self.max_entries = int(max_entries)
        self.keep_outputs = keep_outputs
        self.cell_deg = cell_deg
        self.cell_phase_deg = cell_phase_deg
        self.clock = clock
        self.backend = backend if backend is not None else _CudaBackend(osr)
        self.waiting = collections.deque()
        self.active = []
        self.inflight = collections.deque()
        self.done = []
        self.rejected = []
        self.bytes_in_use = 0
        self.rounds = 0
        self.launches = 0
        self.round_entries = []  # renders per launched round
        self._next_id = 0
        self._ws = [self.backend.workspace(osr_workspace_bytes(osr, self.max_entries))
                    for _ in range(self.max_inflight)]
        self._ws_free = list(range(self.max_inflight))
        self._last_kind = None
        self._plans = None  # per in-flight slot: {kind: plan}, made on first use
        if graphs and hasattr(self.backend, "plan"):
            self._plans = [{} for _ in self._ws]
            for k in range(len(self._ws)):  # Kerr plans up front, off the serving path
                self._plan(k, (osr.SPACETIME_KERR, self.precision))

    # ---- submission and admission ----
    def submit(self, render, arrival=None):
        """Queue a render (a workloads.render dict). Returns its ServedRender.
        Kerr and q-metric renders run at the server's precision (q-metric
        renders in FP64 when it is MIXED); a q-metric disk render (the
        q-metric has no disk model) raises ValueError here, not in a later
        round."""
        osr = self.osr
        if render.get("q") is not None:
            if render["mode"] == "disk":
                raise ValueError("q-metric renders are shadow/lensing renders: the q-metric "
                                 "has no disk model")
            kind = (osr.SPACETIME_QMETRIC,
                    osr.FP64 if self.precision == osr.MIXED else self.precision)
        else:
            kind = (osr.SPACETIME_KERR, self.precision)
        now = self.clock()
        r = ServedRender(self._next_id, render, now if arrival is None else arrival)
        r.kind = kind
        self._next_id += 1
        r.t_submit = now
        if r.bytes > self.hbm_budget:
            self.rejected.append(r)
            return r
        self.waiting.append(r)
        return r

    def _admit(self):
        while self.waiting and self.bytes_in_use + self.waiting[0].bytes <= self.hbm_budget:
            r = self.waiting.popleft()
            rd = r.render
            r.camera = self.backend.camera(rd)
            if r.disk:
                r.r_in = self.backend.resolve_r_in(rd)
                r.r_out = rd["r_out"]
            r.out = self.backend.outputs(r.n_rays, r.disk)
            self.bytes_in_use += r.bytes
            r.t_admit = self.clock()
            self.active.append(r)

    # ---- rounds ----
    def _next_kind(self):
        kinds = []  # kinds with rays left, in order of their oldest such render
        for r in self.active:
            if r.next_ray < r.n_rays and r.kind not in kinds:
                kinds.append(r.kind)
        if not kinds:
            return None
        if len(kinds) > 1 and kinds[0] == self._last_kind:
            return kinds[1]
        return kinds[0]

    def _compose(self):
        kind = self._next_kind()
        budget = self.round_rays
        parts = []
        for r in self.active:  # first pass: a small chunk for every active render
            if budget <= 0 or len(parts) >= self.max_entries:
                break
            if r.kind != kind:
                continue
            left = r.n_rays - r.next_ray
            if left <= 0:
                continue
            n = min(left, self.min_chunk, budget)
            parts.append([r, r.next_ray, n])
            r.next_ray += n
            budget -= n
        for p in parts:  # second pass: the rest to the oldest renders
            if budget <= 0:
                break
            r = p[0]
            extra = min(r.n_rays - r.next_ray, budget)
            if extra > 0 and r.next_ray == p[1] + p[2]:
                p[2] += extra
                r.next_ray += extra
                budget -= extra
        return kind, [tuple(p) for p in parts]

    def _plan(self, k, kind):
        plan = self._plans[k].get(kind)
        if plan is None:
            plan = self.backend.plan(self._ws[k], self.max_entries, spacetime=kind[0],
                                     precision=kind[1], cell_deg=self.cell_deg,
                                     cell_phase_deg=self.cell_phase_deg)
            self._plans[k][kind] = plan
        return plan

    def _launch(self):
        kind, parts = self._compose()
        if not parts:
            return False
        k = self._ws_free.pop()
        entries = []
        for r, first, n in parts:
            entries.append({"camera": r.camera, "disk": r.disk, "r_in": r.r_in, "r_out": r.r_out,
                            "tol": r.tol, "out": r.out, "first_ray": first, "n_rays": n,
                            "l0": r.render.get("l0") if r.disk else None})
            r.chunks.append((first, n))
        if self._plans is not None:
            event = self.backend.launch_plan(self._plan(k, kind), entries)
        else:
            event = self.backend.launch(entries, self._ws[k], precision=kind[1],
                                        cell_deg=self.cell_deg,
                                        cell_phase_deg=self.cell_phase_deg)
        self._last_kind = kind
        self.inflight.append(_Round(event, parts, k, self.clock()))
        self.round_entries.append(len(parts))
        self.rounds += 1
        self.launches += 1
        return True

    def _poll(self):
        progressed = False
        while self.inflight and self.inflight[0].event.query():
            rnd = self.inflight.popleft()
            now = self.clock()
            self._ws_free.append(rnd.ws_index)
            for r, first, n in rnd.parts:
                r.rays_done += n
                if r.rays_done == r.n_rays:
                    r.t_done = now
                    self.active.remove(r)
                    self.done.append(r)
                    self.bytes_in_use -= r.bytes
                    if not self.keep_outputs:
                        r.out = None
                        r.camera = None
            progressed = True
        return progressed

    def step(self):
        """Admit, launch while fewer than max_inflight rounds are queued, and
        retire finished rounds. Returns True when anything happened."""
        progressed = self._poll()
        self._admit()
        while len(self.inflight) < self.max_inflight and self._ws_free:
            if not self._launch():
                break
            progressed = True
        return progressed

    def idle(self):
        return not (self.waiting or self.active or self.inflight)

    def run(self, arrivals, realtime=True, poll_s=2e-4):
        """Serve a list of (arrival_time_s, render). With realtime, each
        render is submitted when the wall clock reaches its arrival time
        (measured from the call); otherwise all are submitted at once."""
        t0 = self.clock()
        pending = collections.deque(sorted(arrivals, key=lambda x: x[0]))
        while pending or not self.idle():
            now = self.clock()
            while pending and (not realtime or pending[0][0] <= now - t0):
                t_arr, rd = pending.popleft()
                self.submit(rd, arrival=t0 + t_arr if realtime else now)
            if not self.step() and poll_s:
                time.sleep(poll_s)
        return summarize(self.done, t0, self.clock(), rejected=len(self.rejected),
                         launches=self.launches)


def shard(arrivals, rank, world):
    """Round-robin share of a render stream (list of (arrival_s, render)) for
    GPU `rank` of `world`: rays are independent, so renders are dealt out
    whole and no data moves between GPUs."""
    ordered = sorted(arrivals, key=lambda x: x[0])
    return [a for k, a in enumerate(ordered) if k % world == rank]


def local_record(done):
    """Per-GPU part of a multi-GPU summary: latencies, rays and time span."""
    if not done:
        return {"latencies": [], "rays": 0, "span": 0.0}
    return {"latencies": [r.t_done - r.arrival for r in done],
            "rays": sum(r.n_rays for r in done),
            "span": max(r.t_done for r in done) - min(r.arrival for r in done)}


def merge_records(records, launches=0):
    """Whole-job summary from the local records of every GPU: percentiles
    over all renders, rays/s = all rays / the longest span."""
    lat = np.array([x for rec in records for x in rec["latencies"]])
    rays = sum(rec["rays"] for rec in records)
    span = max((rec["span"] for rec in records), default=0.0)
    return {"renders": int(lat.size), "rays": rays,
            "p50_latency_s": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_latency_s": float(np.percentile(lat, 99)) if lat.size else None,
            "max_latency_s": float(lat.max()) if lat.size else None,
            "rays_per_s": rays / span if span > 0 else None, "launches": launches}


def osr_workspace_bytes(osr, n):
    return osr.workspace_bytes(n)


def summarize(done, t0, t1, rejected=0, launches=0):
    lat = np.array([r.t_done - r.arrival for r in done]) if done else np.zeros(0)
    rays = sum(r.n_rays for r in done)
    span = (max(r.t_done for r in done) - min(r.arrival for r in done)) if done else 0.0
    return {"renders": len(done), "rejected": rejected, "rays": rays,
            "p50_latency_s": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_latency_s": float(np.percentile(lat, 99)) if lat.size else None,
            "max_latency_s": float(lat.max()) if lat.size else None,
            "rays_per_s": rays / span if span > 0 else None, "wall_s": t1 - t0,
            "launches": launches}


def run_one_per_launch(arrivals, precision=None, realtime=True, clock=time.perf_counter,
                       cell_deg=10.0, cell_phase_deg=0.0, backend=None):
    """Baseline server: renders in arrival order, one plain (non-persistent)
    launch per render, each waited for before the next starts."""
    import paper_2202_00086_gb300 as osr
    backend = backend if backend is not None else _CudaBackend(osr)
    precision = osr.FP64 if precision is None else precision
    t0 = clock()
    done = []
    for t_arr, rd in sorted(arrivals, key=lambda x: x[0]):
        arrival = t0 + t_arr if realtime else clock()
        while realtime and clock() < arrival:
            time.sleep(1e-4)
        r = ServedRender(len(done), rd, arrival)
        r.camera = backend.camera(rd)
        if r.disk:
            r.r_in = backend.resolve_r_in(rd)
            r.r_out = rd["r_out"]
        r.out = backend.outputs(r.n_rays, r.disk)
        backend.single(r, precision=precision, cell_deg=cell_deg, cell_phase_deg=cell_phase_deg)
        r.t_done = clock()
        r.out = None
        done.append(r)
    out = summarize(done, t0, clock(), launches=len(done))
    out["record"] = local_record(done)
    return out


class _CudaBackend:
    """Launches, allocations and events on the current CUDA device."""

    def __init__(self, osr):
        import torch
        self.osr = osr
        self.torch = torch

    def workspace(self, nbytes):
        return self.torch.empty(nbytes, dtype=self.torch.uint8, device="cuda")

    def camera(self, rd):
        return self.osr.Camera.from_render(rd)

    def resolve_r_in(self, rd):
        return self.osr.resolve_r_in(rd)

    def outputs(self, n, disk):
        return self.osr.alloc_outputs(n, fields=self.osr.DISK_FIELDS if disk
                                      else self.osr.SHADOW_FIELDS)

    def launch(self, entries, ws, **opts):
        self.osr.trace_batch(entries, workspace=ws, **opts)
        ev = self.torch.cuda.Event()
        ev.record()
        return ev

    def plan(self, ws, max_entries, **opts):
        return self.osr.BatchPlan(max_entries, workspace=ws, **opts)

    def launch_plan(self, plan, entries):
        plan.launch(entries)
        ev = self.torch.cuda.Event()
        ev.record()
        return ev

    def single(self, r, **opts):
        if r.disk:
            self.osr.render_disk(r.camera, r.r_in, r.r_out, out=r.out, tol=r.tol,
                                 l0=r.render.get("l0"), **opts)
        else:
            self.osr.trace(r.camera, out=r.out, tol=r.tol, **opts)
        self.torch.cuda.synchronize()
