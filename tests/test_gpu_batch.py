"""Batched uneven renders in one persistent launch: the 256-request set
(PCG64 seed 4; sides 128..1024, shadow and Keplerian-disk renders, a, theta0
and r_obs drawn per request), in DF64. Every render is checked against the
oracle on sampled pixels, and the 128^2 renders are bitwise equal to the same
renders traced on their own."""
import time

import numpy as np
import pytest
import torch

import paper_2202_00086_gb300 as osr
from paper_2202_00086_gb300 import workloads

from _parity import assert_parity, compare, gpu_render, oracle_render, oracle_sampled

pytestmark = pytest.mark.gpu


def test_uneven_batch_256():
    rds = workloads.uneven_batch()
    assert len(rds) == 256
    cams = [osr.Camera.from_render(rd) for rd in rds]
    outs = [osr.alloc_outputs(c.n_rays, fields=osr.DISK_FIELDS if rd["mode"] == "disk"
                              else osr.SHADOW_FIELDS) for c, rd in zip(cams, rds)]
    reqs = []
    for c, o, rd in zip(cams, outs, rds):
        disk = rd["mode"] == "disk"
        reqs.append({"camera": c, "disk": disk, "r_in": osr.resolve_r_in(rd) if disk else 0.0,
                     "r_out": rd["r_out"] if disk else 0.0, "tol": rd["tol"], "out": o})
    ws = torch.empty(osr.workspace_bytes(len(reqs)), dtype=torch.uint8, device="cuda")
    stats = osr.new_stats()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    osr.trace_batch(reqs, workspace=ws, precision=osr.DF64, stats=stats,
                    cell_phase_deg=rds[0]["cell_phase_deg"])
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    s = osr.decode_stats(stats)
    n_rays = sum(c.n_rays for c in cams)
    print("uneven batch: %d rays in %.2f s = %.2f Mrays/s" % (n_rays, dt, n_rays / dt / 1e6))
    assert s["rays"] == n_rays and s["status_error"] == 0 and s["status_maxstep"] == 0
    rng = np.random.default_rng(41)
    for k, (rd, o) in enumerate(zip(rds, outs)):
        gpu = {f: v.cpu().numpy() for f, v in o.items()}
        assert int((gpu["status"] == 0).sum()) == 0, k
        if k % 8:
            continue  # oracle check on every 8th render
        pix = np.sort(rng.choice(rd["nx"] * rd["ny"], 24, replace=False))
        ref, band = oracle_sampled(rd, pix)
        rep = compare(rd, gpu, ref, pixels=pix, band=band, precision=osr.DF64)
        print(rep)
        assert_parity(rep)
    small = [k for k, rd in enumerate(rds) if rd["nx"] == 128][:12]
    for k in small:
        alone = gpu_render(rds[k], precision=osr.DF64)
        for f in alone:
            assert np.array_equal(outs[k][f].cpu().numpy(), alone[f]), (k, f)


def _requests(rds, outs, ranges=None):
    reqs = []
    for k, (rd, o) in enumerate(zip(rds, outs)):
        disk = rd["mode"] == "disk"
        q = {"camera": osr.Camera.from_render(rd), "disk": disk,
             "r_in": osr.resolve_r_in(rd) if disk else 0.0,
             "r_out": rd["r_out"] if disk else 0.0, "tol": rd["tol"], "out": o}
        if ranges is not None:
            q["first_ray"], q["n_rays"] = ranges[k]
        reqs.append(q)
    return reqs


def _alloc(rds):
    return [osr.alloc_outputs(rd["nx"] * rd["ny"], fields=osr.DISK_FIELDS if rd["mode"] == "disk"
                              else osr.SHADOW_FIELDS) for rd in rds]


@pytest.mark.parametrize("precision", [osr.FP64, osr.DF64])
def test_batch_plan_graph_matches_trace_batch(precision):
    """Rounds of different sizes and pixel ranges through two CUDA-graph batch
    plans (two rounds in flight on one stream) give bit-identical outputs to
    osiris_trace_batch, and the plan's stats counters add up."""
    rds = workloads.uneven_batch(n=10, seed=9, sides=(16, 32, 48))
    phase = rds[0]["cell_phase_deg"]
    ref = _alloc(rds)
    ws_ref = torch.empty(osr.workspace_bytes(len(rds)), dtype=torch.uint8, device="cuda")
    osr.trace_batch(_requests(rds, ref), workspace=ws_ref, precision=precision,
                    cell_phase_deg=phase)
    got = _alloc(rds)
    stats = osr.new_stats()
    plans = [osr.BatchPlan(8, workspace=torch.empty(osr.workspace_bytes(8), dtype=torch.uint8,
                                                     device="cuda"),
                           precision=precision, cell_phase_deg=phase, stats=stats)
             for _ in range(2)]
    # round k: a pixel range of each render in a sliding window of renders
    n_pix = [rd["nx"] * rd["ny"] for rd in rds]
    done = [0] * len(rds)
    k = 0
    while min(done[i] - n_pix[i] for i in range(len(rds))) < 0:
        idx = [i for i in range(len(rds)) if done[i] < n_pix[i]][: 3 + k % 6]
        ranges = []
        for i in idx:
            n = min(n_pix[i] - done[i], 97 + 211 * (k % 4))
            ranges.append((done[i], n))
            done[i] += n
        reqs = _requests([rds[i] for i in idx], [got[i] for i in idx], ranges)
        plans[k % 2].launch(reqs)
        k += 1
    torch.cuda.synchronize()
    assert k >= 4
    for i, (a, b) in enumerate(zip(ref, got)):
        for f in a:
            assert torch.equal(a[f], b[f]), (i, f)
    s = osr.decode_stats(stats)
    assert s["rays"] == sum(n_pix) and s["status_error"] == 0
    for p in plans:
        p.close()


def test_batch_plan_qmetric_and_errors():
    rds = [workloads.render(0.0, 1000.0, inc, (-8, 8, -8, 8), 12, 10, q=0.3)
           for inc in (40.0, 80.0)]
    ws = torch.empty(osr.workspace_bytes(4), dtype=torch.uint8, device="cuda")
    plan = osr.BatchPlan(4, spacetime=osr.SPACETIME_QMETRIC, workspace=ws,
                         cell_phase_deg=rds[0]["cell_phase_deg"])
    outs = _alloc(rds)
    plan.launch(_requests(rds, outs))
    torch.cuda.synchronize()
    for rd, o in zip(rds, outs):
        alone = gpu_render(rd)
        for f in alone:
            assert np.array_equal(o[f].cpu().numpy(), alone[f]), f
    kerr = workloads.render(0.5, 1000.0, 60.0, (-8, 8, -8, 8), 4, 4)
    with pytest.raises(osr.OsirisError) as e:  # another space-time than the plan's
        plan.launch(_requests([kerr], _alloc([kerr])))
    assert e.value.code == osr.EINVAL
    with pytest.raises(osr.OsirisError) as e:  # more requests than the plan holds
        plan.launch(_requests(rds * 3, _alloc(rds * 3)))
    assert e.value.code == osr.EINVAL
    plan.close()


def test_batch_of_the_maximum_request_count():
    """65536 requests (the most one batch takes), each a one-pixel range of
    one 256^2 render, in one launch: bit-identical to the render traced whole."""
    rd = workloads.render(0.9, 1000.0, 60.0, (-8, 8, -8, 8), 256, 256)
    cam = osr.Camera.from_render(rd)
    out = osr.alloc_outputs(cam.n_rays)
    reqs = [{"camera": cam, "out": out, "tol": rd["tol"], "first_ray": k, "n_rays": 1}
            for k in range(cam.n_rays)]
    assert len(reqs) == 65536
    ws = torch.empty(osr.workspace_bytes(len(reqs)), dtype=torch.uint8, device="cuda")
    stats = osr.new_stats()
    osr.trace_batch(reqs, workspace=ws, stats=stats, cell_deg=rd["cell_deg"],
                    cell_phase_deg=rd["cell_phase_deg"])
    torch.cuda.synchronize()
    assert osr.decode_stats(stats)["rays"] == 65536
    alone = gpu_render(rd)
    for f in alone:
        assert np.array_equal(out[f].cpu().numpy(), alone[f]), f


def test_empty_explicit_states_launch_nothing():
    """Zero explicit rays: the call succeeds, launches nothing and leaves the
    outputs and counters untouched."""
    z = torch.empty(0, dtype=torch.float64, device="cuda")
    st = torch.empty((0, 6), dtype=torch.float64, device="cuda")
    out = osr.alloc_outputs(1)
    before = {f: v.clone() for f, v in out.items()}
    stats = osr.new_stats()
    osr.trace_states(0.5, 1000.0, st, z, z, out=out, stats=stats)
    osr.trace_states(0.5, 1000.0, st, z, z, out=out, stats=stats, precision=osr.DF64)
    torch.cuda.synchronize()
    assert osr.decode_stats(stats)["rays"] == 0
    for f in out:
        assert torch.equal(out[f], before[f]), f
