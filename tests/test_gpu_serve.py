"""The continuous-batching server on the GPU: each render's outputs are the
same (bitwise) alone and in the mix, for shadow and disk renders of different
sizes and tolerances split over several rounds."""
import numpy as np
import pytest
import torch

import paper_2202_00086_gb300 as osr
from paper_2202_00086_gb300 import serve, workloads

pytestmark = pytest.mark.gpu


def _stream(seed=7, n=10):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        side = int(rng.choice([8, 24, 40, 64]))
        a = float(rng.uniform(0.0, 0.998))
        inc = float(rng.uniform(5.0, 85.0))
        tol = 1e-8 if k % 3 == 0 else 1e-10
        if k % 2:
            rd = workloads.render(a, 1000.0, inc, (-25, 25, -25, 25), side, side, mode="disk",
                                  r_in="isco", r_out=20.0, tol=tol)
        else:
            rd = workloads.render(a, 1000.0, inc, (-8, 8, -8, 8), side, side + 2, tol=tol)
        out.append((0.002 * k, rd))
    return out


def _alone(rd, precision, phase):
    cam = osr.Camera.from_render(rd)
    if rd["mode"] == "disk":
        out = osr.render_disk(cam, osr.resolve_r_in(rd), rd["r_out"], tol=rd["tol"],
                              precision=precision, cell_phase_deg=phase)
    else:
        out = osr.trace(cam, tol=rd["tol"], precision=precision, cell_phase_deg=phase)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("precision,overlap,loose", [(osr.DF64, True, None),
                                                     (osr.FP64, True, None),
                                                     (osr.DF64, False, None),
                                                     (osr.DF64, True, osr.MIXED)])
def test_alone_equals_in_the_mix(precision, overlap, loose):
    """Rounds on per-slot streams (overlap: the next round's blocks start in
    the current round's tail) or all on one stream; with a loose precision,
    the renders at tol 1e-8 run in MIXED, the others at the server's."""
    phase = workloads.checker_phase_deg(2202)
    arrivals = _stream()
    srv = serve.RenderServer(precision=precision, round_rays=3000, min_chunk=500,
                             keep_outputs=True, cell_phase_deg=phase, max_inflight=2,
                             overlap=overlap, loose_precision=loose, loose_tol=1e-8)
    summary = srv.run(arrivals, realtime=True)
    torch.cuda.synchronize()
    assert summary["renders"] == len(arrivals)
    assert srv.rounds > 3
    assert max(srv.round_entries) > 1  # renders shared launches
    by_id = {r.rid: r for r in srv.done}
    if loose is not None:
        assert {r.kind[1] for r in srv.done} == {precision, loose}
    for rid, (_, rd) in enumerate(arrivals):
        got = {k: v.cpu().numpy() for k, v in by_id[rid].out.items()}
        ref = _alone(rd, loose if loose is not None and rd["tol"] >= 1e-8 else precision,
                     phase)
        for k in ref:
            assert np.array_equal(got[k], ref[k]), (rid, k)
    assert summary["p99_latency_s"] >= summary["p50_latency_s"] > 0


@pytest.mark.parametrize("graphs", [True, False])
def test_kerr_and_qmetric_in_one_stream(graphs):
    """q-metric renders served next to Kerr renders (both DF64), in rounds of
    one space-time each: every render equals the same render traced alone."""
    phase = workloads.checker_phase_deg(2202)
    rng = np.random.default_rng(3)
    arrivals = []
    for k in range(8):
        side = int(rng.choice([16, 40]))
        if k % 2:
            rd = workloads.render(0.0, 1000.0, float(rng.uniform(20, 85)), (-8, 8, -8, 8), side,
                                  side, q=float(rng.choice([-0.5, 0.1, 0.5])))
        else:
            rd = workloads.render(float(rng.uniform(0, 0.99)), 1000.0, 60.0, (-8, 8, -8, 8),
                                  side, side)
        arrivals.append((0.001 * k, rd))
    srv = serve.RenderServer(round_rays=1500, min_chunk=400, keep_outputs=True,
                             cell_phase_deg=phase, max_inflight=2, graphs=graphs)
    summary = srv.run(arrivals, realtime=True)
    torch.cuda.synchronize()
    assert summary["renders"] == len(arrivals)
    by_id = {r.rid: r for r in srv.done}
    for rid, (_, rd) in enumerate(arrivals):
        got = {k: v.cpu().numpy() for k, v in by_id[rid].out.items()}
        ref = _alone(rd, osr.DF64, phase)
        for k in ref:
            assert np.array_equal(got[k], ref[k]), (rid, k)
