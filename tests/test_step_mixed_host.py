"""One attempt of the MIXED kernels' embedded Runge-Kutta step (step_mixed.cuh:
Cash-Karp 4(5) and Dormand-Prince 5(4), FP32 stage sums over the FP32
evaluation of rhs_f32.cuh at the df64 state plus FP32 increments), compiled as
host C++, against the oracle's FP64 step on the same Kerr state and step
length.

The result carries the FP32 rounding of the derivatives (a few units of
2^-24 of the terms each derivative is summed from, up to ~6e-7 of them next
to the horizon) times the step: measured on these 8,000 attempts, worst
4.9e-7 and median 1.4e-9 of 1 + |y| over the steps the controller accepts
at tol 1e-8 and 1e-7 (error norm at most 1e-7). The error estimate carries a
noise of ~1e-8 h |k| against the oracle's: at error norms of 1e-8 to 1e-7
the two agree to a median of 4 %, 92 % of them within 30 %. A wrong tableau weight or a wrong sign in a stage
difference shows at O(h), a relative error of 1e-3 or more."""
import subprocess

import numpy as np
import pytest

import oracle
from _df_host import build

HARNESS = r"""
#include <cmath>
#include "rhs_f32.cuh"
#include "step_mixed.cuh"
using namespace osiris_impl;
struct HostKerrMixed {  // the Kerr policy of the MIXED kernels, evaluation only
  using Ray = RayF32;
  static void rhs_f(const Ray& K, const PointF32& x, float& dr, float& dth, float& dph,
                    float& dpr, float& dpth, float& twoH) {
    rhs_f32(K, x, dr, dth, dph, dpr, dpth, twoH);
  }
};
static double v(df x) { return (double)x.hi + (double)x.lo; }
template <int I>
static void attempt(const RayF32& k, const StateDF& y, df h, double* out) {
  LaneCacheF32<I> lc;
  lc.reset();
  StateDF o;
  float d[5], twoH;
  rk_step_mixed<HostKerrMixed, I>(k, lc, y, h, o, d, twoH);
  const double r[10] = {v(o.r), v(o.th), v(o.ph), v(o.pr), v(o.pth), d[0], d[1], d[2], d[3], d[4]};
  for (int i = 0; i < 10; ++i) out[i] = r[i];
}
int main() {
  double in[10];  // integrator, a, E, L, r, theta, phi, p_r, p_theta, h
  while (std::fread(in, sizeof in, 1, stdin) == 1) {
    const double a = in[1], E = in[2], L = in[3];
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
    StateDF y;
    y.r = df_from_double(in[4]);
    y.th = df_from_double(in[5]);
    y.ph = df_from_double(in[6]);
    y.pr = df_from_double(in[7]);
    y.pth = df_from_double(in[8]);
    const df h = mk((float)in[9], 0.0f);  // the kernels step with an FP32 length
    double out[10];
    if (in[0] == 0.0)
      attempt<OSIRIS_RKCK45>(k, y, h, out);
    else
      attempt<OSIRIS_RKDP45>(k, y, h, out);
    std::fwrite(out, sizeof out, 1, stdout);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def attempts(tmp_path_factory):
    exe = build(tmp_path_factory, "step_mixed", HARNESS)
    rng = np.random.default_rng(1)
    rows = []
    for integ in (oracle.RKCK45, oracle.RKDP45):
        for a in (0.0, 0.5, 0.9, 0.998):
            r_h = 1.0 + np.sqrt(1.0 - a * a)
            for _ in range(1000):
                r = np.exp(rng.uniform(np.log(1.1 * r_h), np.log(1000.0)))
                h = float(np.float32(r * np.exp(rng.uniform(np.log(1e-3), np.log(0.2)))))
                rows.append([integ, a, 1.0, rng.uniform(-6.0, 6.0), r,
                             rng.uniform(0.1, np.pi - 0.1), 0.3, -rng.uniform(0.0, 1.0),
                             3.0 * rng.normal(), h])
    rows = np.ascontiguousarray(rows, dtype=np.float64)
    p = subprocess.run([str(exe)], input=rows.tobytes(), capture_output=True, check=True)
    out = np.frombuffer(p.stdout, dtype=np.float64).reshape(-1, 10)
    res = []
    for row, o in zip(rows, out):
        integ, a, E, L, r, th, ph, pr, pth, h = row
        y6 = np.array([0.0, r, th, ph, pr, pth])
        y5, d = oracle.rk_step(int(integ), a, y6, E, L, h)
        scale = 1.0 + np.maximum(np.abs(y6[1:]), np.abs(y5[1:]))
        res.append((np.max(np.abs(d[1:]) / scale), o, y5[1:], scale))
    return res


def test_fifth_order_result(attempts):
    kept = [x for x in attempts if x[0] <= 1e-7]
    assert len(kept) > 5000
    errs = np.array([np.max(np.abs(o[:5] - y5) / scale) for _, o, y5, scale in kept])
    assert errs.max() <= 1e-6, errs.max()
    assert np.median(errs) <= 1e-8, np.median(errs)


def test_error_norm_near_the_accept_threshold(attempts):
    kept = [x for x in attempts if 1e-8 <= x[0] <= 1e-7]
    assert len(kept) >= 200
    rel = np.array([abs(np.max(np.abs(o[5:]) / scale) / errn - 1.0)
                    for errn, o, _, scale in kept])
    assert np.median(rel) <= 0.1, np.median(rel)
    assert np.mean(rel <= 0.3) >= 0.85, np.mean(rel <= 0.3)


FSAL_HARNESS = HARNESS[:HARNESS.index("static double v(df x)")] + r"""
static void out5(const StateDF& o, const float* d, double* w) {
  const float f[15] = {o.r.hi, o.r.lo, o.th.hi, o.th.lo, o.ph.hi, o.ph.lo, o.pr.hi, o.pr.lo,
                       o.pth.hi, o.pth.lo, d[0], d[1], d[2], d[3], d[4]};
  for (int i = 0; i < 15; ++i) w[i] = f[i];
}
int main() {
  double in[9];  // a, E, L, r, theta, phi, p_r, p_theta, h
  while (std::fread(in, sizeof in, 1, stdin) == 1) {
    const double a = in[0], E = in[1], L = in[2];
    RayF32 k;
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
    StateDF y;
    y.r = df_from_double(in[3]);
    y.th = df_from_double(in[4]);
    y.ph = df_from_double(in[5]);
    y.pr = df_from_double(in[6]);
    y.pth = df_from_double(in[7]);
    const df h = mk((float)in[8], 0.0f), h2 = mk(0.5f * (float)in[8], 0.0f);
    LaneCacheF32<OSIRIS_RKDP45> lc, fresh;
    lc.reset();
    StateDF o1, o, of;
    float d[5], df_[5], t;
    rk_step_mixed<HostKerrMixed, OSIRIS_RKDP45>(k, lc, y, h, o1, d, t);
    // rejected: retry from y at h/2 with k1 = f(y) kept, and with an empty cache
    double w[60];
    rk_step_mixed<HostKerrMixed, OSIRIS_RKDP45>(k, lc, y, h2, o, d, t);
    fresh.reset();
    rk_step_mixed<HostKerrMixed, OSIRIS_RKDP45>(k, fresh, y, h2, of, df_, t);
    out5(o, d, w);
    out5(of, df_, w + 15);
    // accepted: the next attempt from o with k1 = k7 of this one, and with an empty cache
    lc.accepted();
    rk_step_mixed<HostKerrMixed, OSIRIS_RKDP45>(k, lc, o, h2, o1, d, t);
    fresh.reset();
    rk_step_mixed<HostKerrMixed, OSIRIS_RKDP45>(k, fresh, o, h2, of, df_, t);
    out5(o1, d, w + 30);
    out5(of, df_, w + 45);
    std::fwrite(w, sizeof w, 1, stdout);
  }
  return 0;
}
"""


def test_dormand_prince_cache_is_exact(tmp_path_factory):
    """Dormand-Prince reuses k1 = f(y) after a rejected attempt and k7 = f(o)
    after an accepted one (first same as last): both must give bit for bit
    the attempt that evaluates k1 afresh, since the seventh stage and the
    next first stage evaluate the same point."""
    exe = build(tmp_path_factory, "step_mixed_fsal", FSAL_HARNESS)
    rng = np.random.default_rng(3)
    rows = []
    for a in (0.0, 0.9, 0.998):
        r_h = 1.0 + np.sqrt(1.0 - a * a)
        for _ in range(50):
            r = np.exp(rng.uniform(np.log(1.1 * r_h), np.log(1000.0)))
            h = float(np.float32(r * np.exp(rng.uniform(np.log(1e-3), np.log(0.05)))))
            rows.append([a, 1.0, rng.uniform(-6.0, 6.0), r, rng.uniform(0.1, np.pi - 0.1), 0.3,
                         -rng.uniform(0.0, 1.0), 3.0 * rng.normal(), h])
    rows = np.ascontiguousarray(rows, dtype=np.float64)
    p = subprocess.run([str(exe)], input=rows.tobytes(), capture_output=True, check=True)
    w = np.frombuffer(p.stdout, dtype=np.float64).reshape(-1, 4, 15)
    assert np.all(np.isfinite(w))
    assert np.array_equal(w[:, 0], w[:, 1])  # after a rejection
    assert np.array_equal(w[:, 2], w[:, 3])  # after an acceptance

