"""Host logic of the render server, with a fake backend (no GPU): every pixel
of every admitted render is launched exactly once, rounds respect the ray and
entry budgets, admission respects the HBM budget, and oversize renders are
rejected; Kerr and q-metric renders share the server in rounds of one kind
each."""
import numpy as np

from paper_2202_00086_gb300 import serve, workloads


class FakeEvent:
    def __init__(self, ready_after):
        self.left = ready_after

    def query(self):
        self.left -= 1
        return self.left < 0


class FakeBackend:
    def __init__(self, server_ref, delay=2):
        self.server_ref = server_ref
        self.delay = delay
        self.rounds = []
        self.round_kinds = []  # (set of camera q values, precision) per round
        self.max_bytes_seen = 0

    def workspace(self, nbytes):
        return object()

    def free_bytes(self):
        return 10 << 30

    def camera(self, rd):
        return ("camera", rd["nx"], rd["ny"], rd.get("q"))

    def resolve_r_in(self, rd):
        return 6.0 if rd["r_in"] == "isco" else rd["r_in"]

    def outputs(self, n, disk):
        return {"hits": np.zeros(n, dtype=np.int64)}

    def launch(self, entries, ws, **opts):
        self.rounds.append([(e["first_ray"], e["n_rays"]) for e in entries])
        self.round_kinds.append(({e["camera"][3] for e in entries}, opts.get("precision")))
        for e in entries:
            e["out"]["hits"][e["first_ray"]:e["first_ray"] + e["n_rays"]] += 1
        srv = self.server_ref[0]
        self.max_bytes_seen = max(self.max_bytes_seen, srv.bytes_in_use)
        return FakeEvent(self.delay)


def _server(**kw):
    ref = [None]
    be = FakeBackend(ref)
    srv = serve.RenderServer(backend=be, keep_outputs=True, **kw)
    ref[0] = srv
    return srv, be


def test_every_pixel_once_and_budgets():
    reqs = workloads.uneven_batch(n=40, seed=4, sides=(16, 32, 64, 128))
    budget_rays = 20000
    srv, be = _server(round_rays=budget_rays, min_chunk=1000, max_entries=16,
                      hbm_budget_bytes=3 * 128 * 128 * 66, max_inflight=2)
    summary = srv.run([(0.0, rd) for rd in reqs], realtime=False, poll_s=0)
    assert summary["renders"] == len(reqs) and summary["rejected"] == 0
    for r in srv.done:
        assert np.all(r.out["hits"] == 1)
        # ranges are contiguous and in order
        pos = 0
        for first, n in r.chunks:
            assert first == pos and n > 0
            pos += n
        assert pos == r.n_rays
    for rnd in be.rounds:
        assert sum(n for _, n in rnd) <= budget_rays
        assert len(rnd) <= 16
    assert be.max_bytes_seen <= srv.hbm_budget
    assert srv.bytes_in_use == 0


def test_small_render_finishes_in_its_first_round():
    big = workloads.render(0.5, 1000.0, 60.0, (-8, 8, -8, 8), 512, 512)
    small = workloads.render(0.5, 1000.0, 60.0, (-8, 8, -8, 8), 16, 16)
    srv, be = _server(round_rays=50000, min_chunk=4096, max_inflight=1)
    srv.submit(big, arrival=0.0)
    srv.step()  # the first serving round holds only the big render
    srv.submit(small, arrival=0.0)
    while not srv.idle():
        srv.step()
    small_r = [r for r in srv.done if r.n_rays == 256][0]
    assert len(small_r.chunks) == 1
    # the small render joined the second round, next to the big one
    assert any(len(rnd) == 2 for rnd in be.rounds[1:3])


def test_oversize_render_rejected():
    rd = workloads.render(0.5, 1000.0, 60.0, (-8, 8, -8, 8), 256, 256)
    srv, _ = _server(hbm_budget_bytes=1000)
    r = srv.submit(rd)
    assert r in srv.rejected and srv.idle()


def test_summary_percentiles():
    class R:
        pass
    done = []
    for k in range(100):
        r = R()
        r.arrival, r.t_done, r.n_rays = 0.0, float(k + 1), 10
        done.append(r)
    s = serve.summarize(done, 0.0, 100.0)
    assert abs(s["p50_latency_s"] - 50.5) < 1e-9
    assert abs(s["p99_latency_s"] - 99.01) < 1e-9
    assert s["rays"] == 1000 and abs(s["rays_per_s"] - 10.0) < 1e-12


def test_qmetric_disk_render_is_refused_at_submission():
    import pytest
    srv, be = _server()
    rd = workloads.render(0.0, 1000.0, 60.0, (-25, 25, -25, 25), 16, 16, q=0.3, mode="disk",
                          r_in=6.0, r_out=20.0)
    with pytest.raises(ValueError):
        srv.submit(rd)
    assert srv.idle() and not be.rounds


def test_kerr_and_qmetric_rounds():
    """A launch holds one space-time: every round is all-Kerr or all-q-metric
    (both at the server's precision, DF64 here); while both kinds have rays
    left the rounds alternate, and every pixel is traced once."""
    import paper_2202_00086_gb300 as osr
    rng = np.random.default_rng(9)
    stream = []
    for k in range(24):
        side = int(rng.choice([16, 48, 96]))
        q = float(rng.choice([-0.5, 0.3])) if k % 3 == 1 else None
        stream.append((0.0, workloads.render(0.0 if q is not None else 0.7, 1000.0, 60.0,
                                             (-8, 8, -8, 8), side, side, q=q)))
    srv, be = _server(round_rays=6000, min_chunk=1000, max_inflight=2)
    summary = srv.run(stream, realtime=False, poll_s=0)
    assert summary["renders"] == len(stream)
    for r in srv.done:
        assert np.all(r.out["hits"] == 1)
        assert r.kind == ((osr.SPACETIME_QMETRIC, osr.DF64) if r.render.get("q") is not None
                          else (osr.SPACETIME_KERR, osr.DF64))
    kinds = []
    for qs, prec in be.round_kinds:
        is_q = [q is not None for q in qs]
        assert all(is_q) or not any(is_q)
        assert prec == osr.DF64
        kinds.append(is_q[0])
    assert any(kinds) and not all(kinds)
    # alternation: the q-metric renders are not left until the Kerr ones finish
    last_q = max(i for i, k in enumerate(kinds) if k)
    last_kerr = max(i for i, k in enumerate(kinds) if not k)
    first_switch = next(i for i in range(1, len(kinds)) if kinds[i] != kinds[i - 1])
    assert first_switch == 1
    both_left = min(last_q, last_kerr)
    assert all(kinds[i] != kinds[i + 1] for i in range(both_left))


def test_mixed_server_runs_both_spacetimes_in_mixed():
    import paper_2202_00086_gb300 as osr
    srv, be = _server(precision=osr.MIXED)
    r = srv.submit(workloads.render(0.0, 1000.0, 60.0, (-8, 8, -8, 8), 16, 16, q=0.3))
    k = srv.submit(workloads.render(0.5, 1000.0, 60.0, (-8, 8, -8, 8), 16, 16))
    assert r.kind == (osr.SPACETIME_QMETRIC, osr.MIXED)
    assert k.kind == (osr.SPACETIME_KERR, osr.MIXED)


def test_loose_tolerance_renders_take_the_loose_precision():
    import paper_2202_00086_gb300 as osr
    srv, be = _server(precision=osr.DF64, loose_precision=osr.MIXED, loose_tol=1e-8)
    base = workloads.render(0.5, 1000.0, 60.0, (-8, 8, -8, 8), 16, 16)
    tight = srv.submit(dict(base, tol=1e-10))
    loose = srv.submit(dict(base, tol=1e-8))
    looser = srv.submit(dict(base, tol=1e-6))
    q = srv.submit(dict(workloads.render(0.0, 1000.0, 60.0, (-8, 8, -8, 8), 16, 16, q=0.3),
                        tol=1e-8))
    assert tight.kind == (osr.SPACETIME_KERR, osr.DF64)
    assert loose.kind == looser.kind == (osr.SPACETIME_KERR, osr.MIXED)
    assert q.kind == (osr.SPACETIME_QMETRIC, osr.MIXED)
    while not srv.idle():
        srv.step()
    for r in (tight, loose, looser, q):
        assert r.state == serve.DONE and (r.out["hits"] == 1).all()
    assert {p for _, p in be.round_kinds} == {osr.DF64, osr.MIXED}


class StuckEvent:
    """A round that never completes (a stalled poll made on the host)."""

    def query(self):
        return False


class StuckBackend(FakeBackend):
    def launch(self, entries, ws, **opts):
        super().launch(entries, ws, **opts)
        return StuckEvent()


class TickClock:
    """Deterministic clock: every reading advances it by `dt` seconds."""

    def __init__(self, dt=0.01):
        self.t = 0.0
        self.dt = dt

    def __call__(self):
        self.t += self.dt
        return self.t


def test_cancel_waiting_and_active_renders():
    import paper_2202_00086_gb300 as osr
    big = [workloads.render(0.5, 1000.0, 60.0, (-8, 8, -8, 8), 128, 128) for _ in range(3)]
    srv, be = _server(round_rays=4096, min_chunk=1024, max_inflight=1, max_entries=8)
    rs = [srv.submit(rd, arrival=0.0) for rd in big]
    srv.step()  # admits all three, launches the first round
    assert all(r.state == serve.ACTIVE for r in rs)
    waiting = srv.submit(workloads.render(0.5, 1000.0, 60.0, (-8, 8, -8, 8), 16, 16))
    assert srv.cancel(waiting) and waiting.state == serve.CANCELLED and waiting not in srv.waiting
    launched_before = rs[1].next_ray
    assert 0 < launched_before < rs[1].n_rays
    assert srv.cancel(rs[1])
    assert not srv.cancel(rs[1])  # only once
    while not srv.idle():
        srv.step()
    assert rs[1].state == serve.CANCELLED and rs[1] in srv.cancelled
    assert rs[1].rays_done == launched_before  # no range launched after the cancel
    assert sum(n for first, n in rs[1].chunks) == launched_before
    for r in (rs[0], rs[2]):
        assert r.state == serve.DONE and np.all(r.out["hits"] == 1)
    assert srv.bytes_in_use == 0 and srv.status == osr.OK
    assert not srv.cancel(rs[0])  # already done


def test_stalled_round_times_out_without_waiting_forever():
    import paper_2202_00086_gb300 as osr
    ref = [None]
    be = StuckBackend(ref)
    clock = TickClock(0.01)
    srv = serve.RenderServer(backend=be, keep_outputs=True, clock=clock, stall_timeout_s=1.0,
                             round_rays=2048, min_chunk=512, max_inflight=2)
    ref[0] = srv
    stream = [(0.0, workloads.render(0.5, 1000.0, 60.0, (-8, 8, -8, 8), 64, 64))
              for _ in range(5)]
    summary = srv.run(stream, realtime=False, poll_s=0)
    assert summary["status"] == osr.ETIMEOUT
    assert summary["renders"] == 0
    assert summary["timed_out"] >= 1
    assert summary["timed_out"] + summary["abandoned"] == len(stream)
    assert srv.idle() and srv.bytes_in_use == 0
    n_rounds = len(be.rounds)
    assert srv.submit(stream[0][1]).state == serve.REJECTED  # a stopped server takes nothing
    srv.step()
    assert len(be.rounds) == n_rounds  # and launches nothing
    assert srv.close(timeout_s=0.5) == osr.ETIMEOUT  # the stuck rounds are never waited out
    # the retired renders' output buffers stay held while their rounds may still run
    held = {id(out) for out, _ in srv._held}
    assert len(held) == len(stream) and all(r.out is None for r in srv.failed)
    for rnd in srv.inflight:  # the rounds finally complete: close() releases them
        rnd.event = FakeEvent(0)
    assert srv.close(timeout_s=0.5) == osr.OK and srv._held == []


def test_bounded_wait_for_one_render():
    import paper_2202_00086_gb300 as osr
    srv, be = _server(round_rays=1 << 16, max_inflight=1)
    srv.clock = TickClock(0.001)
    r = srv.submit(workloads.render(0.5, 1000.0, 60.0, (-8, 8, -8, 8), 32, 32))
    assert srv.wait(r, timeout_s=10.0, poll_s=0) == osr.OK and r.state == serve.DONE
    ref = [None]
    stuck = StuckBackend(ref)
    srv2 = serve.RenderServer(backend=stuck, clock=TickClock(0.001), max_inflight=1)
    ref[0] = srv2
    r2 = srv2.submit(workloads.render(0.5, 1000.0, 60.0, (-8, 8, -8, 8), 32, 32))
    assert srv2.wait(r2, timeout_s=0.05, poll_s=0) == osr.ETIMEOUT
    assert r2.state == serve.ACTIVE  # still in flight: nothing was waited for without bound


def test_default_budget_is_a_share_of_free_memory():
    srv, be = _server()
    assert srv.hbm_budget == int(serve.HBM_SHARE * (10 << 30))
    big = workloads.render(0.5, 1000.0, 60.0, (-8, 8, -8, 8), 16384, 16384)  # 11.3 GB of outputs
    assert srv.submit(big).state == serve.REJECTED


class ReorderBackend(FakeBackend):
    """Rounds on different slot streams: every second round completes before
    the round launched ahead of it; records the slot of every launch."""

    def __init__(self, server_ref):
        super().__init__(server_ref)
        self.slots = []

    def launch(self, entries, ws, slot=None, **opts):
        super().launch(entries, ws, **opts)
        self.slots.append(slot)
        return FakeEvent(1 if len(self.slots) % 2 == 0 else 6)


def test_rounds_completing_out_of_order():
    ref = [None]
    be = ReorderBackend(ref)
    srv = serve.RenderServer(backend=be, keep_outputs=True, round_rays=3000, min_chunk=3000,
                             max_inflight=2)
    ref[0] = srv
    reqs = [workloads.render(0.5, 1000.0, 60.0, (-8, 8, -8, 8), 40, 40) for _ in range(6)]
    rs = [srv.submit(rd, arrival=0.0) for rd in reqs]
    order = []
    while not srv.idle():
        srv.step()
        order += [r.rid for r in srv.done if r.rid not in order]
    assert all(r.state == serve.DONE and np.all(r.out["hits"] == 1) for r in rs)
    assert order != sorted(order)  # a later round's render retired first
    assert set(be.slots) == {0, 1}  # each in-flight slot launches on its own stream
    assert srv.bytes_in_use == 0 and not srv.inflight

    ref2 = [None]
    be2 = ReorderBackend(ref2)
    srv2 = serve.RenderServer(backend=be2, keep_outputs=True, round_rays=3000, max_inflight=2,
                              overlap=False)
    ref2[0] = srv2
    srv2.run([(0.0, rd) for rd in reqs], realtime=False, poll_s=0)
    assert set(be2.slots) == {None}  # every round on the current stream
