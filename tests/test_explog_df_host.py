"""The double-float exp and log of the q-metric's double-float evaluation
(explog_df.cuh), compiled as host C++ with the FP32 intrinsics mapped to
plain IEEE single operations, held to 4 units of 2^-48 relative against
mpmath on the arguments the q-metric feeds them and across their range."""
import subprocess

import numpy as np
import pytest

from _df_host import build

HARNESS = r"""
#include "explog_df.cuh"
using namespace osiris_impl;
int main(int argc, char** argv) {
  const bool is_log = argv[1][0] == 'l';
  float v[2];
  while (std::fread(v, sizeof v, 1, stdin) == 1) {
    const df y = is_log ? df_log(mk(v[0], v[1])) : df_exp(mk(v[0], v[1]));
    std::fwrite(&y, sizeof y, 1, stdout);
  }
  return 0;
}
"""

UNIT = 2.0 ** -48


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    exe = build(tmp_path_factory, "explog_df", HARNESS)

    def run(kind, x):
        hi = np.asarray(x, dtype=np.float64).astype(np.float32)
        lo = (x - hi.astype(np.float64)).astype(np.float32)
        a = np.ascontiguousarray(np.stack([hi, lo], 1), dtype=np.float32)
        p = subprocess.run([str(exe), kind], input=a.tobytes(), capture_output=True,
                           check=True)
        return a, np.frombuffer(p.stdout, dtype=np.float32).reshape(-1, 2)
    return run


def _rel_errors(mp, fn, a, out):
    errs = []
    for (h, l), (oh, ol) in zip(a, out):
        w = fn(mp.mpf(float(h)) + mp.mpf(float(l)))
        if w != 0:
            errs.append(float(abs(mp.mpf(float(oh)) + mp.mpf(float(ol)) - w) / abs(w)))
    return np.array(errs)


def test_df_log_bound(harness):
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 120
    rng = np.random.default_rng(1)
    x = np.concatenate([
        rng.uniform(0.0, 1.0, 1500),                                   # f = 1 - 2/r
        1.0 + np.exp(rng.uniform(np.log(1e-14), np.log(1e3), 1500)),   # X >= 1
        1.0 - np.exp(rng.uniform(np.log(1e-14), np.log(0.5), 1500)),   # just below 1
        np.exp(rng.uniform(-60.0, 60.0, 1000)),
    ])
    a, out = harness("l", x)
    err = _rel_errors(mp, mp.log, a, out)
    assert err.max() <= 4 * UNIT, err.max() / UNIT


def test_df_exp_bound(harness):
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 120
    rng = np.random.default_rng(2)
    y = np.concatenate([
        rng.uniform(-69.0, 79.0, 1500),
        rng.uniform(-1.0, 1.0, 1500) * np.exp(rng.uniform(np.log(1e-30), np.log(20.0), 1500)),
        np.arange(-64 * 10, 64 * 10) * (np.log(2.0) / 64.0),   # breakpoints
    ])
    a, out = harness("e", y)
    err = _rel_errors(mp, mp.exp, a, out)
    assert err.max() <= 4 * UNIT, err.max() / UNIT


def test_df_handover(harness):
    """Arguments outside the reduced forms: the FP32 library value, low word 0."""
    with np.errstate(all="ignore"):
        x = np.array([0.0, -1.0, np.inf, np.nan, 1e-35, 1e35])
        a, out = harness("l", x)
        want = np.log(a[:, 0].astype(np.float64))
        assert np.allclose(out[:, 0], want, rtol=2e-7, atol=0, equal_nan=True)
        assert np.all(out[:, 1] == 0.0)
        y = np.array([80.0, -80.0, 100.0, -200.0, np.inf, -np.inf, np.nan])
        a, out = harness("e", y)
        want = np.exp(a[:, 0].astype(np.float64)).astype(np.float32)
        assert np.allclose(out[:, 0], want, rtol=2e-7, atol=0, equal_nan=True)
        assert np.all(out[:, 1] == 0.0)
