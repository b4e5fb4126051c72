"""Continuous-batching render server.

Renders (camera set-ups) arrive over time. The server:
  - admits a waiting render when its output buffers fit in an HBM budget
    (by default 80 % of the device memory free when the server starts;
    outputs stay on the device until the render completes);
  - runs rounds: each round is ONE persistent batched launch over pixel
    ranges of every active render, so renders that arrive while others are on
    the GPU join the next round and their rays share launches with the older
    renders'. With graphs (the default) each in-flight slot owns a batch plan
    (osiris_batch_plan_*): table upload, queue reset and kernel recorded once
    as a CUDA graph, so a round is one graph launch with patched arguments;
    without, a round is one osiris_trace_batch call;
  - keeps up to `max_inflight` rounds in flight, each on the stream of its
    slot (`overlap`, the default), so the GPU never waits for the host
    between rounds and the next round's blocks take the SMs that the
    current round's last, longest rays leave idle (a persistent launch ends
    only when its slowest lane does); with overlap=False every round goes to
    the current stream and runs after the previous one;
  - detects round completion with CUDA events and timestamps each render at
    the completion of its last pixel range.

Round composition: a batched launch holds one space-time and one precision,
so each render has a kind: Kerr renders run at the server's precision, or at
`loose_precision` when one is given and the render's tolerance is at least
`loose_tol` (e.g. MIXED, FP32 stage evaluations and sums, for the renders at 1e-8);
q-metric renders (shadow and lensing; Appendix A) likewise. A round serves one
kind: that of the oldest render with rays left, or the next kind in that
order when the previous round served it, so kinds alternate while several
have work. Within the round every active render of the kind first receives up
to `min_chunk` rays in arrival order (small renders finish in one round),
then the rest of the round budget goes to the oldest of them. Rays are independent, so a
render's outputs are the same whether it runs alone or in a mix (the GPU
tests check this bitwise).

Failure handling (all on the host; nothing waits on the GPU without a
bound):
  - cancel(render): a waiting render is dropped at once; an active one gets no
    further pixel ranges and is retired as cancelled when the ranges already
    launched complete (its outputs are then partial and released);
  - a round that has not completed `stall_timeout_s` after its launch stops
    the server: its renders are retired as timed out (OSIRIS_ETIMEOUT), the
    other active and waiting renders as abandoned, and nothing more is
    launched; run() returns with the status in its summary. The GPU work
    already queued is not recalled (a kernel cannot be interrupted): the
    server keeps its buffers until close() has waited for the stream;
  - wait(render, timeout_s) steps the server until the render is retired or
    the bound runs out, and returns OSIRIS_OK or OSIRIS_ETIMEOUT.

The scheduler is host code; every ray is traced by the CUDA kernels of the
library. For tests without a GPU the launch, allocation and event functions
can be replaced.
"""
import collections
import time

import numpy as np

SHADOW_BYTES_PER_RAY = 42  # status 1, r/theta/phi/max|H| 32, steps 4, cells 4, parity 1
DISK_BYTES_PER_RAY = 66    # + g, intensity, r_hit
HBM_SHARE = 0.8  # default admission budget: this share of the free device memory


# render states
WAITING, ACTIVE, DONE, REJECTED, CANCELLED, TIMED_OUT, ABANDONED = (
    "waiting", "active", "done", "rejected", "cancelled", "timed_out", "abandoned")


class ServedRender:
    __slots__ = ("rid", "render", "arrival", "camera", "disk", "r_in", "r_out", "tol",
                 "n_rays", "next_ray", "rays_done", "out", "bytes", "t_submit", "t_admit",
                 "t_done", "chunks", "kind", "state", "launched")

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
        self.state = WAITING
        self.launched = None  # rays launched when it was cancelled


class _Round:
    __slots__ = ("event", "parts", "ws_index", "t_launch")

    def __init__(self, event, parts, ws_index, t_launch):
        self.event = event
        self.parts = parts
        self.ws_index = ws_index
        self.t_launch = t_launch


class RenderServer:
    def __init__(self, precision=None, round_rays=1 << 21, min_chunk=1 << 14,
                 hbm_budget_bytes=None, max_inflight=2, max_entries=4096,
                 keep_outputs=False, cell_deg=10.0, cell_phase_deg=0.0, backend=None,
                 clock=time.perf_counter, graphs=True, stall_timeout_s=None, overlap=True,
                 loose_precision=None, loose_tol=1e-8):
        import paper_2202_00086_gb300 as osr
        self.osr = osr
        self.precision = osr.DF64 if precision is None else precision
        self.loose_precision = loose_precision
        self.loose_tol = float(loose_tol)
        self.round_rays = int(round_rays)
        self.min_chunk = int(min_chunk)
        self.backend = backend if backend is not None else _CudaBackend(osr)
        if hbm_budget_bytes is None:
            # the renders' device outputs may take this share of the memory that
            # is free when the server starts (the rest is left to the caller)
            hbm_budget_bytes = int(HBM_SHARE * self.backend.free_bytes())
        self.hbm_budget = int(hbm_budget_bytes)
        self.max_inflight = int(max_inflight)
        self.max_entries = int(max_entries)
        self.keep_outputs = keep_outputs
        self.cell_deg = cell_deg
        self.cell_phase_deg = cell_phase_deg
        self.clock = clock
        self.waiting = collections.deque()
        self.active = []
        self.inflight = collections.deque()
        self.done = []
        self.rejected = []
        self.cancelled = []
        self.failed = []  # timed out or abandoned after a stalled round
        self.stall_timeout_s = stall_timeout_s
        self.overlap = bool(overlap)
        self.status = osr.OK
        self._held = []  # buffers of renders retired while their rounds may still run
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
        Renders run at the server's precision, or at its loose precision when
        their tolerance is loose enough; a q-metric disk render (the q-metric
        has no disk model) raises ValueError here, not in a later round."""
        osr = self.osr
        prec = self.precision
        if self.loose_precision is not None and render["tol"] >= self.loose_tol:
            prec = self.loose_precision
        if render.get("q") is not None:
            if render["mode"] == "disk":
                raise ValueError("q-metric renders are shadow/lensing renders: the q-metric "
                                 "has no disk model")
            kind = (osr.SPACETIME_QMETRIC, prec)
        else:
            kind = (osr.SPACETIME_KERR, prec)
        now = self.clock()
        r = ServedRender(self._next_id, render, now if arrival is None else arrival)
        r.kind = kind
        self._next_id += 1
        r.t_submit = now
        if r.bytes > self.hbm_budget or self.status != osr.OK:
            r.state = REJECTED
            self.rejected.append(r)
            return r
        self.waiting.append(r)
        return r

    def cancel(self, r):
        """Cancel a submitted render. Returns True if it was waiting or
        active (it is then retired as cancelled, at once or when its
        launched pixel ranges complete), False if it had already left."""
        if r.state == WAITING:
            self.waiting.remove(r)
            r.state = CANCELLED
            r.t_done = self.clock()
            self.cancelled.append(r)
            return True
        if r.state != ACTIVE or r.launched is not None:
            return False
        r.launched = r.next_ray
        r.next_ray = r.n_rays  # no further pixel ranges
        if r.rays_done == r.launched:
            self._retire(r, CANCELLED, self.clock())
        return True

    def _retire(self, r, state, now):
        r.state = state
        r.t_done = now
        self.active.remove(r)
        self.bytes_in_use -= r.bytes
        (self.done if state == DONE else
         self.cancelled if state == CANCELLED else self.failed).append(r)
        if state in (TIMED_OUT, ABANDONED):
            # launched ranges may still be running: their output buffers stay
            # allocated until close() has seen every round complete
            self._held.append((r.out, r.camera))
        if not self.keep_outputs or state != DONE:
            r.out = None
            r.camera = None

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
            r.state = ACTIVE
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
        slot = k if self.overlap else None  # None: the current stream
        if self._plans is not None:
            event = self.backend.launch_plan(self._plan(k, kind), entries, slot=slot)
        else:
            event = self.backend.launch(entries, self._ws[k], slot=slot, precision=kind[1],
                                        cell_deg=self.cell_deg,
                                        cell_phase_deg=self.cell_phase_deg)
        self._last_kind = kind
        self.inflight.append(_Round(event, parts, k, self.clock()))
        self.round_entries.append(len(parts))
        self.rounds += 1
        self.launches += 1
        return True

    def _finished_rounds(self):
        """In-flight rounds whose event has completed, oldest first (rounds on
        different slot streams may complete out of launch order)."""
        return [rnd for rnd in self.inflight if rnd.event.query()]

    def _poll(self):
        progressed = False
        for rnd in self._finished_rounds():
            self.inflight.remove(rnd)
            now = self.clock()
            self._ws_free.append(rnd.ws_index)
            for r, first, n in rnd.parts:
                r.rays_done += n
                if r.launched is not None:
                    if r.rays_done == r.launched:
                        self._retire(r, CANCELLED, now)
                elif r.rays_done == r.n_rays:
                    self._retire(r, DONE, now)
            progressed = True
        if (self.inflight and self.stall_timeout_s is not None
                and self.clock() - self.inflight[0].t_launch > self.stall_timeout_s):
            self._stall()
            progressed = True
        return progressed

    def _stall(self):
        """The oldest round missed its bound: retire its renders as timed out,
        every other render as abandoned, and launch nothing more."""
        now = self.clock()
        self.status = self.osr.ETIMEOUT
        stalled = {id(r) for r, _, _ in self.inflight[0].parts}
        for r in list(self.active):
            self._retire(r, TIMED_OUT if id(r) in stalled else ABANDONED, now)
        while self.waiting:
            r = self.waiting.popleft()
            r.state = ABANDONED
            r.t_done = now
            self.failed.append(r)

    def step(self):
        """Admit, launch while fewer than max_inflight rounds are queued, and
        retire finished rounds. Returns True when anything happened. After a
        stalled round (status OSIRIS_ETIMEOUT) it launches nothing."""
        progressed = self._poll()
        if self.status != self.osr.OK:
            return progressed
        self._admit()
        while len(self.inflight) < self.max_inflight and self._ws_free:
            if not self._launch():
                break
            progressed = True
        return progressed

    def idle(self):
        if self.status != self.osr.OK:
            return True
        return not (self.waiting or self.active or self.inflight)

    def wait(self, r, timeout_s, poll_s=2e-4):
        """Step the server until render r has left (done, cancelled or
        failed) or timeout_s has passed. Returns OSIRIS_OK or OSIRIS_ETIMEOUT
        (the render then stays queued or in flight)."""
        t0 = self.clock()
        while r.state in (WAITING, ACTIVE):
            if self.clock() - t0 > timeout_s:
                return self.osr.ETIMEOUT
            if not self.step() and poll_s:
                time.sleep(poll_s)
        return self.osr.ETIMEOUT if r.state in (TIMED_OUT, ABANDONED) else self.osr.OK

    def close(self, timeout_s=None):
        """Wait (bounded when timeout_s is given) for every launched round,
        then release the buffers of renders retired while their rounds were
        still running; returns OSIRIS_OK or OSIRIS_ETIMEOUT (the buffers are
        then kept)."""
        t0 = self.clock()
        while self.inflight:
            finished = self._finished_rounds()
            for rnd in finished:
                self.inflight.remove(rnd)
            if finished:
                continue
            if timeout_s is not None and self.clock() - t0 > timeout_s:
                return self.osr.ETIMEOUT
            time.sleep(2e-4)
        self._held = []
        return self.osr.OK

    def run(self, arrivals, realtime=True, poll_s=2e-4):
        """Serve a list of (arrival_time_s, render). With realtime, each
        render is submitted when the wall clock reaches its arrival time
        (measured from the call); otherwise all are submitted at once. Stops
        early when a round stalls (summary "status" OSIRIS_ETIMEOUT)."""
        t0 = self.clock()
        self.t0 = t0
        pending = collections.deque(sorted(arrivals, key=lambda x: x[0]))
        while (pending or not self.idle()) and self.status == self.osr.OK:
            now = self.clock()
            while pending and (not realtime or pending[0][0] <= now - t0):
                t_arr, rd = pending.popleft()
                self.submit(rd, arrival=t0 + t_arr if realtime else now)
            if not self.step() and poll_s:
                time.sleep(poll_s)
        out = summarize(self.done, t0, self.clock(), rejected=len(self.rejected),
                        launches=self.launches)
        out.update(status=self.status, cancelled=len(self.cancelled),
                   timed_out=sum(r.state == TIMED_OUT for r in self.failed),
                   abandoned=sum(r.state == ABANDONED for r in self.failed) + len(pending))
        return out


def shard(arrivals, rank, world):
    """Round-robin share of a render stream (list of (arrival_s, render)) for
    GPU `rank` of `world`: rays are independent, so renders are dealt out
    whole and no data moves between GPUs."""
    ordered = sorted(arrivals, key=lambda x: x[0])
    return [a for k, a in enumerate(ordered) if k % world == rank]


def local_record(done, t0=None):
    """Per-GPU part of a multi-GPU summary: latencies, rays and time span;
    with t0 (the clock reading the stream's arrival times count from), also
    each render's arrival time, its ray count and the time its last pixel
    range completed, both relative to t0."""
    if not done:
        return {"latencies": [], "rays": 0, "span": 0.0, "arrivals": [], "done_at": [],
                "n_rays": []}
    rec = {"latencies": [r.t_done - r.arrival for r in done],
           "rays": sum(r.n_rays for r in done),
           "span": max(r.t_done for r in done) - min(r.arrival for r in done)}
    if t0 is not None:
        rec["arrivals"] = [r.arrival - t0 for r in done]
        rec["done_at"] = [r.t_done - t0 for r in done]
        rec["n_rays"] = [r.n_rays for r in done]
    return rec


def latency_windows(records, duration_s, width_s=10.0):
    """Latency percentiles of the renders that arrived in each window of
    width_s seconds of the stream (records: local_record(done, t0) of every
    GPU), the growth of p99 from the first third of the stream to the last,
    and the backlog: rays that had arrived but were not yet complete when
    the last arrival came (duration_s)."""
    arr = np.array([a for rec in records for a in rec.get("arrivals", [])])
    lat = np.array([x for rec in records for x in rec["latencies"]])
    done_at = np.array([a for rec in records for a in rec.get("done_at", [])])
    n_rays = np.array([a for rec in records for a in rec.get("n_rays", [])])
    if arr.size == 0:
        return {"windows": [], "p99_growth": None, "backlog_rays_at_last_arrival": None}
    windows = []
    w0 = 0.0
    while w0 < duration_s:
        m = (arr >= w0) & (arr < w0 + width_s)
        if m.any():
            windows.append({"from_s": w0, "renders": int(m.sum()),
                            "p50_latency_s": float(np.percentile(lat[m], 50)),
                            "p99_latency_s": float(np.percentile(lat[m], 99))})
        w0 += width_s
    first = arr < duration_s / 3
    last = arr >= 2 * duration_s / 3
    growth = None
    if first.any() and last.any():
        growth = float(np.percentile(lat[last], 99) / np.percentile(lat[first], 99))
    backlog = int(n_rays[(arr <= duration_s) & (done_at > duration_s)].sum())
    return {"windows": windows, "p99_growth": growth, "backlog_rays_at_last_arrival": backlog}


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
        self._streams = {}

    def _stream(self, slot):
        """The stream of an in-flight slot (None: the current stream). A slot
        stream first waits for the work queued so far on the current stream,
        so a round never overtakes what the caller queued before it."""
        cur = self.torch.cuda.current_stream()
        if slot is None:
            return cur
        s = self._streams.get(slot)
        if s is None:
            s = self._streams[slot] = self.torch.cuda.Stream()
        s.wait_stream(cur)
        return s

    def workspace(self, nbytes):
        return self.torch.empty(nbytes, dtype=self.torch.uint8, device="cuda")

    def free_bytes(self):
        """Device memory free now (cudaMemGetInfo), plus what torch's caching
        allocator holds but does not use."""
        free, _ = self.torch.cuda.mem_get_info()
        cached = self.torch.cuda.memory_reserved() - self.torch.cuda.memory_allocated()
        return free + cached

    def camera(self, rd):
        return self.osr.Camera.from_render(rd)

    def resolve_r_in(self, rd):
        return self.osr.resolve_r_in(rd)

    def outputs(self, n, disk):
        return self.osr.alloc_outputs(n, fields=self.osr.DISK_FIELDS if disk
                                      else self.osr.SHADOW_FIELDS)

    def launch(self, entries, ws, slot=None, **opts):
        s = self._stream(slot)
        self.osr.trace_batch(entries, workspace=ws, stream=s, **opts)
        ev = self.torch.cuda.Event()
        ev.record(s)
        return ev

    def plan(self, ws, max_entries, **opts):
        return self.osr.BatchPlan(max_entries, workspace=ws, **opts)

    def launch_plan(self, plan, entries, slot=None):
        s = self._stream(slot)  # a plan belongs to one slot, so to one stream
        plan.launch(entries, stream=s)
        ev = self.torch.cuda.Event()
        ev.record(s)
        return ev

    def single(self, r, **opts):
        if r.disk:
            self.osr.render_disk(r.camera, r.r_in, r.r_out, out=r.out, tol=r.tol,
                                 l0=r.render.get("l0"), **opts)
        else:
            self.osr.trace(r.camera, out=r.out, tol=r.tol, **opts)
        self.torch.cuda.synchronize()
