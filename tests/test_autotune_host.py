"""Autotuner selection and cache logic (no GPU: a fake timer)."""
import os

import pytest

from paper_2202_00086_gb300 import autotune


def test_choose_fastest_with_ties():
    t = {(128, 0): 1.0, (64, 2): 0.8, (256, 0): 0.8, (64, 0): 0.8}
    assert autotune.choose(t) == (64, 0)
    t4 = {(128, 0, 2, 1): 0.5, (128, 0, 0, 0): 0.5, (128, 0, 1, 4): 0.6}
    assert autotune.choose(t4) == (128, 0, 0, 0)  # ties: the library's default distribution
    with pytest.raises(ValueError):
        autotune.choose({})


def test_two_stage_search_with_fake_timer_writes_cache(tmp_path):
    """Stage 1 picks the launch shape with the library's default work
    distribution; stage 2 times every granularity at that shape only."""
    path = os.path.join(tmp_path, "tune.json")
    shape_cost = {(64, 0): 3.0, (128, 0): 2.0, (128, 3): 1.5, (256, 1): 4.0}
    gran_cost = {(0, 0): 0.0, (2, 1): -0.2, (2, 16): -0.1, (8, 32): 0.3}
    calls = []

    def timer(b, k, r, f):
        calls.append((b, k, r, f))
        return shape_cost[(b, k)] + gran_cost[(r, f)]

    best, timings = autotune.autotune(precision=2, integrator=1, cands=list(shape_cost),
                                      grans=list(gran_cost), cache_path=path, timer=timer)
    assert best == (128, 3, 2, 1)
    assert [c for c in calls if c[2:] != (0, 0)] == [(128, 3, 2, 1), (128, 3, 2, 16),
                                                   (128, 3, 8, 32)]
    assert len(timings) == len(shape_cost) + len(gran_cost) - 1
    opts = autotune.tuned_opts(2, 1, cache_path=path, device_name="test-device")
    assert opts == {"block_size": 128, "blocks_per_sm": 3, "rays_per_lane": 2,
                    "refill_lanes": 1}
    assert autotune.tuned_opts(0, 0, cache_path=path, device_name="test-device") == {}
