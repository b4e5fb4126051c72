"""The double-float (df64) arithmetic of the DF64 kernels (df64.cuh), compiled
as host C++, against mpmath: sine and cosine over the angles rays take
(relative accuracy kept next to the poles and the equator, where the
reduction subtracts a multiple of pi/2 exactly, down to values of 1e-9), the
reciprocal of a normalised pair, and products and sums. The bound is a few
units of 2^-48 (48 significand bits)."""
import subprocess

import numpy as np
import pytest

from _df_host import build

HARNESS = r"""
#include "df64.cuh"
using namespace osiris_impl;
int main(int argc, char** argv) {
  const char op = argv[1][0];
  float v[4];
  while (std::fread(v, sizeof v, 1, stdin) == 1) {
    const df a = mk(v[0], v[1]), b = mk(v[2], v[3]);
    df r0 = mk(0.0f, 0.0f), r1 = mk(0.0f, 0.0f);
    if (op == 's') df_sincos(a, r0, r1);
    else if (op == 'r') r0 = df_rcp(a);
    else if (op == 'm') r0 = df_mul(a, b);
    else if (op == 'a') r0 = df_add(a, b);
    const float out[4] = {r0.hi, r0.lo, r1.hi, r1.lo};
    std::fwrite(out, sizeof out, 1, stdout);
  }
  return 0;
}
"""

UNIT = 2.0 ** -48


def _split(x):
    x = np.asarray(x, dtype=np.float64)
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    return hi, lo


@pytest.fixture(scope="module")
def df64(tmp_path_factory):
    exe = build(tmp_path_factory, "df64", HARNESS)

    def run(op, a, b=None):
        ah, al = _split(a)
        bh, bl = _split(np.zeros_like(np.asarray(a, dtype=np.float64)) if b is None else b)
        inp = np.ascontiguousarray(np.stack([ah, al, bh, bl], 1), dtype=np.float32)
        p = subprocess.run([str(exe), op], input=inp.tobytes(), capture_output=True,
                           check=True)
        out = np.frombuffer(p.stdout, dtype=np.float32).reshape(-1, 4).astype(np.float64)
        exact_in = ah.astype(np.float64) + al.astype(np.float64)
        exact_b = bh.astype(np.float64) + bl.astype(np.float64)
        return exact_in, exact_b, out[:, 0] + out[:, 1], out[:, 2] + out[:, 3]
    return run


def _mp():
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 120
    return mp


def test_sincos(df64):
    mp = _mp()
    rng = np.random.default_rng(1)
    th = np.concatenate([
        rng.uniform(-0.5, np.pi + 0.5, 3000),
        rng.uniform(-1.0, 1.0, 500) * np.exp(rng.uniform(np.log(1e-12), 0.0, 500)),  # pole
        np.pi + rng.uniform(-1.0, 1.0, 500) * np.exp(rng.uniform(np.log(1e-12), 0.0, 500)),
        np.pi / 2 + rng.uniform(-1.0, 1.0, 500) * np.exp(rng.uniform(np.log(1e-12), 0.0, 500)),
    ])
    x, _, s, c = df64("s", th)
    worst_abs = worst_rel = worst_tiny = 0.0
    for xi, si, ci in zip(x, s, c):
        for got, want in ((si, mp.sin(mp.mpf(float(xi)))), (ci, mp.cos(mp.mpf(float(xi))))):
            e = float(abs(got - want))
            worst_abs = max(worst_abs, e)
            if abs(want) >= 1e-9:
                worst_rel = max(worst_rel, e / float(abs(want)))
            else:
                worst_tiny = max(worst_tiny, e)
    assert worst_abs <= 4 * UNIT, worst_abs / UNIT
    # next to the poles and the equator the reduction subtracts k pi/2 exactly,
    # so sin (cos) keeps its relative accuracy; pi/2 is held to 76 bits, an
    # absolute 4e-23 for k = 2, which bounds values closer than 1e-9 to zero
    assert worst_rel <= 1e-13, worst_rel
    assert worst_tiny <= 1e-21, worst_tiny


def test_reciprocal_of_normalised_pairs(df64):
    mp = _mp()
    rng = np.random.default_rng(2)
    b = np.exp(rng.uniform(np.log(1e-12), np.log(1e12), 4000)) * rng.choice([-1.0, 1.0], 4000)
    x, _, r, _ = df64("r", b)
    err = max(float(abs(mp.mpf(float(ri)) * mp.mpf(float(xi)) - 1)) for xi, ri in zip(x, r))
    assert err <= 4 * UNIT, err / UNIT


def test_products_and_sums(df64):
    mp = _mp()
    rng = np.random.default_rng(3)
    a = rng.uniform(-1.0, 1.0, 3000) * np.exp(rng.uniform(-20.0, 20.0, 3000))
    b = rng.uniform(-1.0, 1.0, 3000) * np.exp(rng.uniform(-20.0, 20.0, 3000))
    x, y, p, _ = df64("m", a, b)
    errm = max(float(abs(mp.mpf(float(pi)) / (mp.mpf(float(xi)) * mp.mpf(float(yi))) - 1))
               for xi, yi, pi in zip(x, y, p))
    assert errm <= 4 * UNIT, errm / UNIT
    # sums of like-signed terms (no cancellation: the relative bound applies)
    x, y, s, _ = df64("a", np.abs(a), np.abs(b))
    erra = max(float(abs(mp.mpf(float(si)) / (mp.mpf(float(xi)) + mp.mpf(float(yi))) - 1))
               for xi, yi, si in zip(x, y, s))
    assert erra <= 4 * UNIT, erra / UNIT
