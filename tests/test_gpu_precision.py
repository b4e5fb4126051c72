"""Parity of the reduced-precision paths with the FP64 oracle.

DF64 (double-float stage evaluations, df64 state) is held to the same bar as
the FP64 kernels. MIXED (FP32 stage evaluations and sums around a df64 state) is
held to its stated error bound: flags identical outside the oracle's band,
redshift g within 1e-5 and coordinates within 1e-5 (relative) of the oracle
at 1e-10, when MIXED runs at tolerances of 1e-7 to 1e-8.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2202_00086_gb300 as osr
from paper_2202_00086_gb300 import workloads

from _parity import assert_parity, compare, gpu_render, oracle_render, oracle_sampled

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("a", workloads.KERR_SPINS)
@pytest.mark.parametrize("inc", workloads.KERR_INCLINATIONS)
def test_df64_kerr_subsampled(a, inc):
    rd = workloads.render(a, 1000.0, inc, (-8, 8, -8, 8), 32, 32)
    rep = compare(rd, gpu_render(rd, precision=osr.DF64), oracle_render(rd), precision=osr.DF64)
    print(rep)
    assert_parity(rep)
    assert rep["theta_max_rel"] < 1e-9 and rep["phi_max_rel"] < 1e-9


def test_df64_disks():
    for rd in (workloads.schwarzschild_disk(side=64),
               workloads.render(0.9, 1000.0, 60.0, (-25, 25, -25, 25), 40, 40, mode="disk",
                                r_in="isco", r_out=20.0)):
        rep = compare(rd, gpu_render(rd, precision=osr.DF64), oracle_render(rd),
                      precision=osr.DF64)
        print(rep)
        assert_parity(rep)
        assert rep["n_disk"] > 100 and rep["g_max_rel"] < 1e-9


def test_df64_persistent_matches_plain_and_ragged():
    rd = workloads.render(0.998, 1000.0, 17.0, (-8, 8, -8, 8), 37, 29)
    a = gpu_render(rd, precision=osr.DF64)
    b = gpu_render(rd, precision=osr.DF64, persistent=True, block_size=64)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    assert_parity(compare(rd, a, oracle_render(rd), precision=osr.DF64))


def test_df64_max_steps_and_states():
    rd = workloads.render(0.9, 1000.0, 60.0, (-8, 8, -8, 8), 16, 16)
    gpu = gpu_render(rd, precision=osr.DF64, max_steps=40)
    ref = oracle_render(rd, max_steps=40)
    assert np.array_equal(gpu["status"], ref["status"])
    assert (ref["status"] == osr.STATUS_MAXSTEP).sum() > 0


@pytest.mark.parametrize("precision", [osr.FP64, osr.DF64])
def test_full_size_batch_sampled(precision):
    """The 12-render 1024^2 Kerr set in one batched launch, exactly as the
    benchmark times it (FP64 headline and DF64 variant), 50 sampled pixels per
    render checked against the oracle."""
    rds = workloads.kerr_shadow_ring_set(1024)
    cams = [osr.Camera.from_render(rd) for rd in rds]
    outs = [osr.alloc_outputs(c.n_rays) for c in cams]
    ws = torch.empty(osr.workspace_bytes(len(cams)), dtype=torch.uint8, device="cuda")
    osr.trace_batch([{"camera": c, "out": o} for c, o in zip(cams, outs)], workspace=ws,
                    precision=precision, tol=1e-10, cell_deg=rds[0]["cell_deg"],
                    cell_phase_deg=rds[0]["cell_phase_deg"])
    torch.cuda.synchronize()
    rng = np.random.default_rng(12)
    for rd, o in zip(rds, outs):
        gpu = {k: v.cpu().numpy() for k, v in o.items()}
        pix = np.sort(rng.choice(1024 * 1024, 50, replace=False))
        ref, band = oracle_sampled(rd, pix)
        rep = compare(rd, gpu, ref, pixels=pix, band=band, precision=precision)
        print(rep)
        assert_parity(rep)


@pytest.mark.parametrize("tol", [1e-7, 1e-8])
def test_mixed_error_bound(tol):
    rd = dict(workloads.schwarzschild_disk(side=48))
    rd["tol"] = tol
    ref = oracle_render(dict(rd, tol=1e-10))
    rep = compare(rd, gpu_render(rd, precision=osr.MIXED), ref, coord_rtol=1e-5, g_rtol=1e-5,
                  precision=osr.MIXED)
    print(rep)
    assert_parity(rep)
    assert rep["n_disk"] > 150


@pytest.mark.parametrize("a,inc", [(0.998, 60.0), (0.5, 17.0), (0.0, 85.0)])
def test_mixed_error_bound_kerr_shadow(a, inc):
    rd = dict(workloads.render(a, 1000.0, inc, (-8, 8, -8, 8), 40, 40), tol=1e-8)
    ref = oracle_render(dict(rd, tol=1e-10))
    rep = compare(rd, gpu_render(rd, precision=osr.MIXED), ref, coord_rtol=1e-5,
                  precision=osr.MIXED)
    print(rep)
    assert_parity(rep)
    st = np.asarray(ref["status"])
    assert (st == oracle.STATUS_CAPTURED).sum() > 100 and (st == oracle.STATUS_ESCAPED).sum() > 100


def test_mixed_full_size_sampled():
    """A 1024^2 Kerr render in MIXED at tol 1e-8, persistent launch, sampled
    against the oracle at 1e-10 with the oracle's band."""
    rd = dict(workloads.kerr_shadow_ring_set(1024)[3 * 3 + 1], tol=1e-8)
    gpu = gpu_render(rd, precision=osr.MIXED, persistent=True)
    rng = np.random.default_rng(23)
    pix = np.sort(rng.choice(1024 * 1024, 200, replace=False))
    ref, band = oracle_sampled(dict(rd, tol=1e-10), pix)
    rep = compare(rd, gpu, ref, pixels=pix, band=band, coord_rtol=1e-5, precision=osr.MIXED)
    print(rep)
    assert_parity(rep)


def test_df64_tracks_H_like_fp64():
    """The double-float kernel reports the same constraint error as the FP64
    kernel: per-ray max |H| of a Kerr render (light, H0 = 0), and of unit-mass
    particles (H0 = -1/2, where |H - H0| ~ 1e-10 sits far below FP32's
    resolution of H0 itself)."""
    import math
    rd = workloads.render(0.998, 1000.0, 60.0, (-8, 8, -8, 8), 40, 40)
    g64 = gpu_render(rd)
    h64 = g64["max_abs_H"]
    hdf = gpu_render(rd, precision=osr.DF64)["max_abs_H"]
    assert np.all(np.isfinite(hdf)) and np.all(hdf > 0)
    assert hdf.max() == pytest.approx(h64.max(), rel=0.2)
    assert 0.9 < np.median(hdf / h64) < 1.1
    # captured rays end next to the horizon, where Delta nearly cancels: the
    # double-float arithmetic must keep their |H| at the FP64 kernel's level
    cap = g64["status"] == osr.STATUS_CAPTURED
    assert cap.sum() > 100
    assert 0.8 < np.median(hdf[cap] / h64[cap]) < 1.25
    # unit-mass particles launched outwards from r = 30 in Kerr a = 0.9
    a, r = 0.9, 30.0
    rng = np.random.default_rng(8)
    th = rng.uniform(0.4, math.pi - 0.4, 64)
    E = np.full(64, 1.2)
    L = rng.uniform(-4.0, 4.0, 64)
    s2 = np.sin(th) ** 2
    Sig, Del = r * r + a * a * (1 - s2), r * r - 2 * r + a * a
    A = (r * r + a * a) ** 2 - a * a * Del * s2
    gtt, gtp = -A / (Sig * Del), -2 * a * r / (Sig * Del)
    gpp, grr = (Del - a * a * s2) / (Sig * Del * s2), Del / Sig
    pr = np.sqrt((-1.0 - (gtt * E * E - 2 * gtp * E * L + gpp * L * L)) / grr)
    st = np.zeros((64, 6))
    st[:, 1], st[:, 2], st[:, 4] = r, th, pr
    args = (torch.tensor(st, device="cuda"), torch.tensor(E, device="cuda"),
            torch.tensor(L, device="cuda"))
    res = {p: osr.trace_states(a, 1000.0, *args, mass2=1.0, precision=p)["max_abs_H"]
           .cpu().numpy() for p in (osr.FP64, osr.DF64)}
    assert np.all(res[osr.DF64] > 0) and np.all(res[osr.FP64] > 0)
    assert res[osr.DF64].max() == pytest.approx(res[osr.FP64].max(), rel=0.5)
