"""Autotuner selection and cache logic (no GPU: a fake timer)."""
import os

import pytest

from paper_2202_00086_gb300 import autotune


def test_choose_fastest_with_ties():
    t = {(128, 0): 1.0, (64, 2): 0.8, (256, 0): 0.8, (64, 0): 0.8}
    assert autotune.choose(t) == (64, 0)
    with pytest.raises(ValueError):
        autotune.choose({})


def test_autotune_with_fake_timer_writes_cache(tmp_path):
    path = os.path.join(tmp_path, "tune.json")
    cost = {(64, 0): 3.0, (128, 0): 2.0, (128, 3): 1.5, (256, 1): 4.0}
    best, timings = autotune.autotune(precision=2, integrator=1, cands=list(cost),
                                      cache_path=path, timer=lambda b, k: cost[(b, k)])
    assert best == (128, 3) and timings == cost
    opts = autotune.tuned_opts(2, 1, cache_path=path, device_name="test-device")
    assert opts == {"block_size": 128, "blocks_per_sm": 3}
    assert autotune.tuned_opts(0, 0, cache_path=path, device_name="test-device") == {}
