"""The FP32 evaluation of Hamilton's equations used by the MIXED kernels
(rhs_f32.cuh: Kerr in the separated form of the FP64 kernels), compiled as
host C++, against the oracle's component-form equations at random
phase-space points, off the constraint surface and down to 1.02 horizon
radii, and its sine and cosine against numpy next to the poles.

FP32 carries 24 significand bits, so each derivative must agree with the
oracle to 2e-6 of the size of the terms it is summed from (the largest
derivative, and (u^2 + p_r^2) r / Sigma with u = P / Delta, the terms that
cancel in p_r' next to the horizon), and r' and theta' (no cancellation)
to 2e-6 relative: which holds next to the horizon only because Delta is
formed as (r - r+)(r - r-) from both words of the df64 radius (in FP32,
r^2 - 2r + a^2 keeps no correct digit at 1.02 r+ for a = 0.998). sin and cos
must keep 1e-6 relative accuracy from 1e-8 to 1e-5 away from the poles and
the equator, where the quadrant reduction works from both words of theta
(its absolute floor, the FP32 rounding of theta.lo - k P2, is ~1e-14; a ray
passes within 1e-8 of a pole almost never). Measured worst: 6.4e-7 of the
terms, 2.8e-7 relative."""
import subprocess

import numpy as np
import pytest

import oracle
from _df_host import build

HARNESS = r"""
#include <cstdlib>
#include "rhs_f32.cuh"
using namespace osiris_impl;
// The point (r, theta, p_r, p_theta) as a stage input of the MIXED stepper:
// df64 bases r - dr and theta - dth plus the FP32 increments dr, dth (both
// exact floats, -0 for a point given by its base alone).
static PointF32 point(const double* v, double dr, double dth) {
  PointF32 x;
  x.r = df_from_double(v[0] - dr);
  x.th = df_from_double(v[1] - dth);
  x.dr = (float)dr;
  x.dth = (float)dth;
  x.pr = (float)v[2];
  x.pth = (float)v[3];
  return x;
}
int main(int argc, char** argv) {
  const char op = argv[1][0];
  double in[9];  // 'e': a, E, L, r, theta, p_r, p_theta, dr, dth; 's': theta, dth
  const int n = op == 'e' ? 9 : 2;
  while (std::fread(in, sizeof(double) * n, 1, stdin) == 1) {
    if (op == 's') {
      float s, c;
      sincos_f32(df_from_double(in[0] - in[1]), (float)in[1], s, c);
      const double out[2] = {s, c};
      std::fwrite(out, sizeof out, 1, stdout);
      continue;
    }
    const double a = in[0], E = in[1], L = in[2];
    RayF32 k;  // ray constants formed as the MIXED kernels form them
    k.a = (float)a;
    k.a2 = (float)(a * a);
    k.aE = (float)(a * E);
    k.aL = (float)(a * L);
    k.E = (float)E;
    k.L = (float)L;
    k.twoE = (float)(2.0 * E);
    const double sq = std::sqrt(std::fmax(0.0, 1.0 - a * a));
    k.rp = df_from_double(1.0 + sq);
    k.rm = (float)(1.0 - sq);
    k.twoH0 = 0.0f;
    float d[5], twoH;
    rhs_f32(k, point(in + 3, in[7], in[8]), d[0], d[1], d[2], d[3], d[4], twoH);
    const double out[6] = {d[0], d[1], d[2], d[3], d[4], twoH};
    std::fwrite(out, sizeof out, 1, stdout);
  }
  return 0;
}
"""


def _split(rows, seed):
    """Append the increments (dr, dth) of the stage-input form: a quarter of
    the points given by their base alone (-0), the rest split into a base and
    an FP32 increment of up to 5 % of r and 0.3 rad."""
    rng = np.random.default_rng(seed)
    rows = np.asarray(rows, dtype=np.float64)
    n = len(rows)
    dr = np.float32(rows[:, 3] * rng.uniform(-0.05, 0.05, n)).astype(np.float64)
    dth = np.float32(rng.uniform(-0.3, 0.3, n)).astype(np.float64)
    base = rng.uniform(size=n) < 0.25
    dr[base] = -0.0
    dth[base] = -0.0
    return np.column_stack([rows, dr, dth])


@pytest.fixture(scope="module")
def dev(tmp_path_factory):
    exe = build(tmp_path_factory, "rhs_f32", HARNESS)

    def run(op, rows, width):
        inp = np.ascontiguousarray(rows, dtype=np.float64)
        p = subprocess.run([str(exe), op], input=inp.tobytes(), capture_output=True, check=True)
        return np.frombuffer(p.stdout, dtype=np.float64).reshape(-1, width)
    return run


def _points(n, seed):
    rng = np.random.default_rng(seed)
    rows = []
    for a in (0.0, 0.5, 0.9, 0.998):
        r_min = 1.02 * (1.0 + np.sqrt(1.0 - a * a))
        for _ in range(n):
            rows.append([a, 1.0, rng.uniform(-8.0, 8.0),
                         np.exp(rng.uniform(np.log(r_min), np.log(1000.0))),
                         rng.uniform(0.05, np.pi - 0.05), 2.0 * rng.normal(), 5.0 * rng.normal()])
    return np.array(rows)


def _errors(rows, out):
    worst_terms = worst_rel = 0.0
    for row, o in zip(rows, out):
        a, E, L, r, th, pr, pth = row
        y6 = np.array([0.0, r, th, 0.0, pr, pth])
        dy = oracle.rhs_sp(oracle.KERR, y6, E, L, a=a)
        delta = r * r - 2.0 * r + a * a
        sigma = r * r + a * a * np.cos(th) ** 2
        u = ((r * r + a * a) * E - a * L) / delta
        scale = np.abs(dy[1:]).max() + (u * u + pr * pr) * max(r, 1.0) / sigma
        err = np.abs(o[:5] - dy[1:])
        worst_terms = max(worst_terms, err.max() / scale)
        worst_rel = max(worst_rel, err[0] / abs(dy[1]), err[1] / abs(dy[2]))
    return worst_terms, worst_rel


def test_kerr_rhs_f32_against_oracle(dev):
    rows = _points(150, 11)
    worst_terms, worst_rel = _errors(rows, dev("e", _split(rows, 21), 6))
    assert worst_terms <= 2e-6 and worst_rel <= 2e-6, (worst_terms, worst_rel)


def test_kerr_rhs_f32_next_to_the_horizon(dev):
    rng = np.random.default_rng(12)
    rows = []
    for a in (0.0, 0.9, 0.998):
        r_h = 1.0 + np.sqrt(1.0 - a * a)
        for f in (1.0001, 1.001, 1.01, 1.02):
            for _ in range(20):
                rows.append([a, 1.0, rng.uniform(-4.0, 4.0), f * r_h, rng.uniform(0.3, 2.8),
                             rng.normal(), 3.0 * rng.normal()])
    rows = np.array(rows)
    worst_terms, worst_rel = _errors(rows, dev("e", _split(rows, 22), 6))
    assert worst_terms <= 2e-6 and worst_rel <= 2e-6, (worst_terms, worst_rel)


def test_sincos_f32_next_to_poles_and_equator(dev):
    rng = np.random.default_rng(13)
    centres = (0.0, 0.5 * np.pi, np.pi, 1.5 * np.pi, -0.5 * np.pi)
    th = np.concatenate([c + np.exp(rng.uniform(np.log(1e-8), np.log(1e-5), 60))
                         * rng.choice([-1.0, 1.0], 60) for c in centres])
    th = np.concatenate([th, rng.uniform(-np.pi, 2.0 * np.pi, 300)])
    dth = np.float32(rng.uniform(-0.3, 0.3, len(th))).astype(np.float64)
    dth[::4] = -0.0
    out = dev("s", np.column_stack([th, dth]), 2)
    rel_s = np.abs(out[:, 0] - np.sin(th)) / np.abs(np.sin(th))
    rel_c = np.abs(out[:, 1] - np.cos(th)) / np.abs(np.cos(th))
    assert rel_s.max() <= 1e-6 and rel_c.max() <= 1e-6, (rel_s.max(), rel_c.max())


QHARNESS = r"""
#include "rhs_f32.cuh"
using namespace osiris_impl;
int main() {
  double in[9];  // q, E, L, r, theta, p_r, p_theta, dr, dth (as in HARNESS)
  while (std::fread(in, sizeof in, 1, stdin) == 1) {
    const double q = in[0], E = in[1], L = in[2];
    RayQF32 k;  // ray constants formed as the MIXED kernels form them
    k.E = (float)E;
    k.L = (float)L;
    k.q = (float)q;
    k.kap = (float)(q * (2.0 + q));
    k.nq1 = (float)(-(1.0 + q));
    k.E2 = (float)(E * E);
    k.twoH0 = 0.0f;
    float d[5], twoH;
    PointF32 x;
    x.r = df_from_double(in[3] - in[7]);
    x.th = df_from_double(in[4] - in[8]);
    x.dr = (float)in[7];
    x.dth = (float)in[8];
    x.pr = (float)in[5];
    x.pth = (float)in[6];
    rhs_q_f32(k, x, d[0], d[1], d[2], d[3], d[4], twoH);
    const double out[6] = {d[0], d[1], d[2], d[3], d[4], twoH};
    std::fwrite(out, sizeof out, 1, stdout);
  }
  return 0;
}
"""


def test_qmetric_rhs_q_f32_against_oracle(tmp_path_factory):
    """The q-metric in FP32 (MIXED) against the oracle's component form, down to
    r = 2.02: every derivative within 2e-6 of the largest one at that point,
    r' and theta' within 2e-6 relative (measured 7.7e-7 and 3.4e-7 with the
    host's exp and log; the GPU's FP32 exp and log intrinsics add a few 1e-7
    to the powers f^q and X^k, inside the bound)."""
    exe = build(tmp_path_factory, "rhs_q_f32", QHARNESS)
    rng = np.random.default_rng(14)
    rows = []
    for q in (-0.5, 0.1, 0.5):
        for _ in range(150):
            rows.append([q, 1.0, rng.uniform(-8.0, 8.0),
                         np.exp(rng.uniform(np.log(2.02), np.log(1000.0))),
                         rng.uniform(0.05, np.pi - 0.05), 2.0 * rng.normal(), 5.0 * rng.normal()])
    rows = np.array(rows)
    p = subprocess.run([str(exe)], input=np.ascontiguousarray(_split(rows, 23)).tobytes(),
                       capture_output=True, check=True)
    out = np.frombuffer(p.stdout, dtype=np.float64).reshape(-1, 6)
    worst_terms = worst_rel = 0.0
    for row, o in zip(rows, out):
        q, E, L, r, th, pr, pth = row
        y6 = np.array([0.0, r, th, 0.0, pr, pth])
        dy = oracle.rhs_sp(oracle.QMETRIC, y6, E, L, q=q)
        err = np.abs(o[:5] - dy[1:])
        worst_terms = max(worst_terms, err.max() / np.abs(dy[1:]).max())
        worst_rel = max(worst_rel, err[0] / abs(dy[1]), err[1] / abs(dy[2]))
    assert worst_terms <= 2e-6 and worst_rel <= 2e-6, (worst_terms, worst_rel)
