"""The autotuner on the GPU: it times real launches, picks one of the
candidates, and the tuned launch shape gives the same outputs (rays are
independent of the launch shape)."""
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
    best, timings = autotune.autotune(osr.DF64, 0, renders=rds, cands=cands, cache_path=path)
    assert best in cands and len(timings) == len(cands)
    assert all(t > 0 for t in timings.values())
    opts = autotune.tuned_opts(osr.DF64, 0, cache_path=path)
    assert opts["block_size"] == best[0]
    a = gpu_render(rds[1], precision=osr.DF64, persistent=True, **opts)
    b = gpu_render(rds[1], precision=osr.DF64)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
