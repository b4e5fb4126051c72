"""One attempt of the DF64 kernels' double-float embedded Runge-Kutta step
(step_df.cuh: Cash-Karp 4(5) and Dormand-Prince 5(4) with their tableaus as
float pairs), compiled as host C++, against the oracle's step on the same
Kerr state and step length.

The DF64 stepper sums the O(h) part of each stage input in FP32 by design.
That perturbs the stages by about (h/T)^2 6e-8 relative, which is negligible
for the result at the step lengths the controller accepts (error norm at most
~1e-9 at tol 1e-10; measured worst 1.3e-11 of 1 + |y|), but it leaves the error
estimate, a difference of O((h/T)^5), with a floor near 1e-12 of 1 + |y|; the
error sum itself is an FP32 sum of exact stage differences. At the accept
threshold the DF64 error norm agrees with the oracle's to about a percent
(measured on these 39 attempts: median 1.0 %, worst 11 %), which is why the
DF64 kernels take the oracle's accept/reject decision on most but not all
steps. A wrong tableau constant would show at O(h): in the fifth-order
result, or through the error weights no longer summing to zero."""
import subprocess

import numpy as np
import pytest

import oracle
from _df_host import build

HARNESS = r"""
#include "rhs_df.cuh"
#include "step_df.cuh"
using namespace osiris_impl;
struct HostKerr {  // the Kerr policy of the DF64 kernels, evaluation only
  using Ray = RayDF;
  static void rhs(const Ray& K, df r, df th, df pr, df pth, df& dr, df& dth, df& dph, df& dpr,
                  df& dpth, float& twoH) {
    rhs_df(K, r, th, pr, pth, dr, dth, dph, dpr, dpth, twoH);
  }
};
static double v(df x) { return (double)x.hi + (double)x.lo; }
template <int I>
static void attempt(const RayDF& k, const StateDF& y, df h, double* out) {
  LaneCacheDF<I> lc;
  lc.reset();
  StateDF o;
  float d[5], twoH;
  rk_step_df<HostKerr, I>(k, lc, y, h, o, d, twoH);
  const double r[10] = {v(o.r), v(o.th), v(o.ph), v(o.pr), v(o.pth), d[0], d[1], d[2], d[3], d[4]};
  for (int i = 0; i < 10; ++i) out[i] = r[i];
}
int main() {
  double in[10];  // integrator, a, E, L, r, theta, phi, p_r, p_theta, h
  while (std::fread(in, sizeof in, 1, stdin) == 1) {
    const double a = in[1], E = in[2], L = in[3];
    RayDF k;
    k.a = df_from_double(a);
    k.a2 = df_from_double(a * a);
    k.aE = df_from_double(a * E);
    k.aL = df_from_double(a * L);
    k.E = df_from_double(E);
    k.L = df_from_double(L);
    k.twoE = df_scale(k.E, 2.0f);
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
    exe = build(tmp_path_factory, "step_df", HARNESS)
    rng = np.random.default_rng(1)
    rows = []
    for integ in (oracle.RKCK45, oracle.RKDP45):
        for a in (0.0, 0.5, 0.9, 0.998):
            r_h = 1.0 + np.sqrt(1.0 - a * a)
            for _ in range(200):
                r = np.exp(rng.uniform(np.log(1.1 * r_h), np.log(1000.0)))
                h = float(np.float32(r * np.exp(rng.uniform(np.log(1e-4), np.log(0.05)))))
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
        res.append((np.max(np.abs(d[1:]) / scale), o, y5[1:], d[1:], scale))
    return res


def test_fifth_order_result(attempts):
    kept = [x for x in attempts if x[0] <= 1e-9]
    assert len(kept) > 800
    for errn, o, y5, d, scale in kept:
        assert np.max(np.abs(o[:5] - y5) / scale) <= 1e-10, (errn, o[:5], y5)


def test_error_norm_at_the_accept_threshold(attempts):
    kept = [x for x in attempts if 1e-10 <= x[0] <= 1e-9]
    assert len(kept) >= 20
    for errn, o, y5, d, scale in kept:
        errn_df = np.max(np.abs(o[5:]) / scale)
        assert abs(errn_df / errn - 1.0) <= 0.15, (errn, errn_df)


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
    RayDF k;
    k.a = df_from_double(a);
    k.a2 = df_from_double(a * a);
    k.aE = df_from_double(a * E);
    k.aL = df_from_double(a * L);
    k.E = df_from_double(E);
    k.L = df_from_double(L);
    k.twoE = df_scale(k.E, 2.0f);
    k.twoH0 = 0.0f;
    StateDF y;
    y.r = df_from_double(in[3]);
    y.th = df_from_double(in[4]);
    y.ph = df_from_double(in[5]);
    y.pr = df_from_double(in[6]);
    y.pth = df_from_double(in[7]);
    const df h = mk((float)in[8], 0.0f), h2 = mk(0.5f * (float)in[8], 0.0f);
    LaneCacheDF<OSIRIS_RKDP45> lc, fresh;
    lc.reset();
    StateDF o1, o, of;
    float d[5], df_[5], t;
    rk_step_df<HostKerr, OSIRIS_RKDP45>(k, lc, y, h, o1, d, t);
    double w[60];
    // rejected: retry from y at h/2 with k1 = f(y) kept, and with an empty cache
    rk_step_df<HostKerr, OSIRIS_RKDP45>(k, lc, y, h2, o, d, t);
    fresh.reset();
    rk_step_df<HostKerr, OSIRIS_RKDP45>(k, fresh, y, h2, of, df_, t);
    out5(o, d, w);
    out5(of, df_, w + 15);
    // accepted: the next attempt from o with k1 = k7 of this one, and with an empty cache
    lc.accepted();
    rk_step_df<HostKerr, OSIRIS_RKDP45>(k, lc, o, h2, o1, d, t);
    fresh.reset();
    rk_step_df<HostKerr, OSIRIS_RKDP45>(k, fresh, o, h2, of, df_, t);
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
    next first stage evaluate the same df64 point."""
    exe = build(tmp_path_factory, "step_df_fsal", FSAL_HARNESS)
    rng = np.random.default_rng(3)
    rows = []
    for a in (0.0, 0.9, 0.998):
        r_h = 1.0 + np.sqrt(1.0 - a * a)
        for _ in range(50):
            r = np.exp(rng.uniform(np.log(1.1 * r_h), np.log(1000.0)))
            h = float(np.float32(r * np.exp(rng.uniform(np.log(1e-4), np.log(0.05)))))
            rows.append([a, 1.0, rng.uniform(-6.0, 6.0), r, rng.uniform(0.1, np.pi - 0.1), 0.3,
                         -rng.uniform(0.0, 1.0), 3.0 * rng.normal(), h])
    rows = np.ascontiguousarray(rows, dtype=np.float64)
    p = subprocess.run([str(exe)], input=rows.tobytes(), capture_output=True, check=True)
    w = np.frombuffer(p.stdout, dtype=np.float64).reshape(-1, 4, 15)
    assert np.all(np.isfinite(w))
    assert np.array_equal(w[:, 0], w[:, 1])  # after a rejection
    assert np.array_equal(w[:, 2], w[:, 3])  # after an acceptance

