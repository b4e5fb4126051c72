"""The table-driven exp and log of the q-metric evaluation (explog.cuh),
compiled as host C++ and held to their error bound: within 2 ulp of the
exact value (mpmath at 200 bits; measured worst cases 1.0 ulp for exp and 2.0
for log on ten times this test's sample, where log F/2 and log1p(u) partly
cancel, the same as with the all-FP64 series) on sampled arguments, within
2.5 ulp of libm on a million arguments over the ranges the q-metric feeds them
(f = 1 - 2/r in (0, 1), X = 1 + sin^2/(r^2 - 2r) >= 1, and q log f,
k log X), and equal to libm where they hand over to it (0, negatives,
subnormals, infinities, NaN, |y| >= 700)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from _df_host import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2202_00086_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <vector>
#include "explog.cuh"
using namespace osiris_explog;
int main(int argc, char** argv) {
  const bool is_log = argv[1][0] == 'l';
  std::vector<double> x;
  double v;
  while (std::fread(&v, sizeof v, 1, stdin) == 1) x.push_back(v);
  for (double a : x) {
    const double y = is_log ? log_tab(a, kLg) : exp_tab(a, kT2);
    std::fwrite(&y, sizeof y, 1, stdout);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    # the FP32 intrinsics of the double-float corrections map to IEEE single
    # operations (the shims of the other host builds)
    exe = build(tmp_path_factory, "explog", HARNESS)

    def run(kind, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        p = subprocess.run([str(exe), kind], input=x.tobytes(), capture_output=True,
                           check=True)
        return np.frombuffer(p.stdout, dtype=np.float64)
    return run


def _ulp_err(got, want):
    return np.abs(got - want) / np.spacing(np.abs(want))


def _log_args(rng, n):
    return np.concatenate([
        rng.uniform(0.0, 1.0, n),                         # f near and far from the horizon
        np.exp(rng.uniform(np.log(1e-12), 0.0, n)),
        1.0 + np.exp(rng.uniform(np.log(1e-15), np.log(1e6), n)),   # X
        1.0 - np.exp(rng.uniform(np.log(1e-16), np.log(0.5), n)),   # just below 1
        np.exp(rng.uniform(-690.0, 690.0, n)),
        np.ldexp(1.0, np.arange(-1000, 1001)),
        np.nextafter(np.ldexp(1.0, np.arange(-999, 1001)), 0.0),
    ])


def _exp_args(rng, n):
    return np.concatenate([
        rng.uniform(-699.0, 699.0, n),
        rng.uniform(-1.0, 1.0, n) * np.exp(rng.uniform(np.log(1e-300), np.log(30.0), n)),
        np.arange(-700 * 64, 700 * 64) * (np.log(2.0) / 64.0),   # at the breakpoints
        (np.arange(-700 * 64, 700 * 64) + 0.5) * (np.log(2.0) / 64.0),  # mid-way
    ])


def test_log_near_libm(harness):
    x = _log_args(np.random.default_rng(3), 200_000)
    err = _ulp_err(harness("l", x), np.log(x))
    assert err.max() <= 2.5, (err.max(), x[err.argmax()])


def test_exp_near_libm(harness):
    y = _exp_args(np.random.default_rng(4), 200_000)
    want = np.exp(y)
    ok = want > np.finfo(np.float64).tiny  # below: subnormal results, none here
    err = _ulp_err(harness("e", y)[ok], want[ok])
    assert err.max() <= 2.5, (err.max(), y[ok][err.argmax()])


def test_exp_log_within_2ulp_of_exact(harness):
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 200
    rng = np.random.default_rng(5)
    x = _log_args(rng, 300)
    y = _exp_args(rng, 300)[:3000]
    gl, ge = harness("l", x), harness("e", y)
    for a, g in zip(x, gl):
        want = float(mp.log(mp.mpf(float(a))))
        if want != 0.0:
            assert abs(g - want) <= 2 * np.spacing(abs(want)), (a, g, want)
        else:
            assert g == 0.0
    for a, g in zip(y, ge):
        want = float(mp.exp(mp.mpf(float(a))))
        assert abs(g - want) <= 2 * np.spacing(abs(want)), (a, g, want)


def test_qmetric_powers(harness):
    """f^q and X^k as the q-metric evaluation forms them, against libm's pow."""
    rng = np.random.default_rng(6)
    r = 2.0 + np.exp(rng.uniform(np.log(1e-9), np.log(1e6), 100_000))
    s2 = np.sin(rng.uniform(1e-8, np.pi - 1e-8, r.size)) ** 2
    f = (r - 2.0) / r
    X = 1.0 + s2 / (r * (r - 2.0))
    for q in (-0.9, -0.5, 0.1, 0.5, 0.9):
        k = q * (2.0 + q)
        fq = harness("e", q * harness("l", f))
        Xk = harness("e", k * harness("l", X))
        # an absolute error in y = q log f (2 ulp of log f, 0.5 ulp of the
        # product) is a relative error of exp(y), on top of exp's own 2 ulp
        # and pow's rounding: about 3e-16 (1 + |y|) measured, 6e-16 allowed
        tol_f = 6e-16 * (1.0 + np.abs(q * np.log(f)))
        tol_X = 6e-16 * (1.0 + np.abs(k * np.log(X)))
        assert np.all(np.abs(fq / f ** q - 1.0) <= tol_f), q
        assert np.all(np.abs(Xk / X ** k - 1.0) <= tol_X), q


def test_handover_to_libm(harness):
    with np.errstate(all="ignore"):
        x = np.array([0.0, -0.0, -1.0, -np.inf, np.inf, np.nan, 5e-324, 1e-310,
                      np.ldexp(1.0, -1001), np.ldexp(1.0, 1001), 1.7e308])
        gl, wl = harness("l", x), np.log(x)
        assert np.array_equal(gl, wl, equal_nan=True)
        y = np.array([700.0, -700.0, 709.7, -745.0, -1000.0, 1000.0, np.inf, -np.inf, np.nan])
        ge, we = harness("e", y), np.exp(y)
        assert np.array_equal(ge, we, equal_nan=True)
