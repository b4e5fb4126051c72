"""The autotuner on the GPU: it times real launches over launch shapes and
work granularities (rays per lane, refill lanes), picks one of the
candidates, and the tuned launch gives the same outputs (rays are
independent of how they are distributed); so does every granularity, in
plain and persistent launches, FP64 and DF64."""
import os

import numpy as np
import pytest
import torch

import paper_2202_00086_gb300 as osr
from paper_2202_00086_gb300 import autotune, workloads

from _parity import gpu_render

pytestmark = pytest.mark.gpu


def test_autotune_small_sample(tmp_path):
    path = os.path.join(tmp_path, "tune.json")
    rds = [workloads.render(a, 1000.0, 60.0, (-8, 8, -8, 8), 48, 48) for a in (0.0, 0.9)]
    cands = [(64, 0), (128, 0), (128, 2), (256, 1)]
    grans = [(0, 0), (2, 4), (4, 32)]
    best, timings = autotune.autotune(osr.DF64, 0, renders=rds, cands=cands, grans=grans,
                                      cache_path=path)
    assert best[:2] in cands and best[2:] in grans
    assert len(timings) == len(cands) + len(grans) - 1
    assert all(t > 0 for t in timings.values())
    opts = autotune.tuned_opts(osr.DF64, 0, cache_path=path)
    assert (opts["block_size"], opts["rays_per_lane"]) == (best[0], best[2])
    a = gpu_render(rds[1], precision=osr.DF64, persistent=True, **opts)
    b = gpu_render(rds[1], precision=osr.DF64)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("precision", [osr.FP64, osr.DF64, osr.MIXED])
def test_granularity_does_not_change_outputs(precision):
    """37x29 render (ragged against every block and claim size): plain
    launches with 1, 3 and 8 rays per thread and persistent launches with
    several claim sizes and refill thresholds give bit-identical outputs."""
    rd = workloads.render(0.998, 1000.0, 60.0, (-8, 8, -8, 8), 37, 29)
    ref = gpu_render(rd, precision=precision)
    for kw in (dict(rays_per_lane=3), dict(rays_per_lane=8, block_size=32),
               dict(persistent=True, rays_per_lane=2, refill_lanes=1),
               dict(persistent=True, rays_per_lane=5, refill_lanes=16, block_size=64),
               dict(persistent=True, rays_per_lane=1, refill_lanes=32)):
        got = gpu_render(rd, precision=precision, **kw)
        for k in ref:
            assert np.array_equal(ref[k], got[k]), (kw, k)
    with pytest.raises(osr.OsirisError):
        gpu_render(rd, rays_per_lane=65)
    with pytest.raises(osr.OsirisError):
        gpu_render(rd, persistent=True, refill_lanes=33)
