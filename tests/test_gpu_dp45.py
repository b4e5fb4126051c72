"""Dormand-Prince 5(4) on the GPU against the oracle's Dormand-Prince path
(same parity bar as Cash-Karp), in FP64 and DF64, including the
first-same-as-last cache across accepts, rejects, surface location and
disk misses."""
import numpy as np
import pytest
import torch

import oracle
import paper_2202_00086_gb300 as osr
from paper_2202_00086_gb300 import workloads

from _parity import assert_parity, compare, gpu_render, oracle_render, oracle_sampled

pytestmark = pytest.mark.gpu
DP = osr.RKDP45


@pytest.mark.parametrize("precision", [osr.FP64, osr.DF64])
@pytest.mark.parametrize("a,inc", [(0.0, 17.0), (0.5, 60.0), (0.9, 90.0), (0.998, 60.0),
                                   (0.998, 17.0)])
def test_dp45_kerr_subsampled(precision, a, inc):
    rd = workloads.render(a, 1000.0, inc, (-8, 8, -8, 8), 32, 32)
    ref = oracle_render(rd, integrator=oracle.RKDP45)
    rep = compare(rd, gpu_render(rd, precision=precision, integrator=DP), ref,
                  precision=precision)
    print(rep)
    assert_parity(rep)


@pytest.mark.parametrize("precision", [osr.FP64, osr.DF64])
def test_dp45_disks(precision):
    for rd in (workloads.schwarzschild_disk(side=48),
               workloads.render(0.9, 1000.0, 60.0, (-25, 25, -25, 25), 40, 40, mode="disk",
                                r_in="isco", r_out=20.0)):
        ref = oracle_render(rd, integrator=oracle.RKDP45)
        rep = compare(rd, gpu_render(rd, precision=precision, integrator=DP), ref,
                      precision=precision)
        print(rep)
        assert_parity(rep)
        assert rep["n_disk"] > 100


@pytest.mark.parametrize("precision", [osr.FP64, osr.DF64])
def test_dp45_persistent_matches_plain(precision):
    rd = workloads.render(0.998, 1000.0, 60.0, (-8, 8, -8, 8), 37, 29)
    a = gpu_render(rd, precision=precision, integrator=DP)
    b = gpu_render(rd, precision=precision, integrator=DP, persistent=True, block_size=64)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_dp45_keeps_H_smaller_on_gpu():
    rd = workloads.render(0.98, 1000.0, 90.0, (-8, 8, -8, 8), 48, 48)
    ck = gpu_render(rd)
    dp = gpu_render(rd, integrator=DP)
    cap = ck["status"] == osr.STATUS_CAPTURED
    assert dp["max_abs_H"][cap].mean() < ck["max_abs_H"][cap].mean() / 5


def test_dp45_full_size_sampled():
    rd = workloads.kerr_shadow_ring_set(1024)[3 * 3 + 1]
    gpu = gpu_render(rd, precision=osr.DF64, integrator=DP, persistent=True)
    rng = np.random.default_rng(21)
    pix = np.sort(rng.choice(1024 * 1024, 300, replace=False))
    ref, band = oracle_sampled(rd, pix, integrator=oracle.RKDP45)
    rep = compare(rd, gpu, ref, pixels=pix, band=band, precision=osr.DF64)
    print(rep)
    assert_parity(rep)


def test_dp45_mixed_error_bound():
    """Dormand-Prince with FP32 stage evaluations (MIXED) at tol 1e-8 against
    the oracle's Dormand-Prince at 1e-10: the MIXED error bound."""
    rd = dict(workloads.render(0.9, 1000.0, 60.0, (-8, 8, -8, 8), 40, 40), tol=1e-8)
    ref = oracle_render(dict(rd, tol=1e-10), integrator=oracle.RKDP45)
    rep = compare(rd, gpu_render(rd, precision=osr.MIXED, integrator=DP), ref, coord_rtol=1e-5,
                  precision=osr.MIXED)
    print(rep)
    assert_parity(rep)
