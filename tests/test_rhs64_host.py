"""The FP64 kernels' evaluation of Hamilton's equations (trace_device.cuh:
rhs64 for Kerr in the separated form, rhs_q64 for the q-metric in the
collected form) and its helpers, compiled as host C++ (a block of one thread,
the tables filled as the kernels fill them; the FP32 reciprocal seed is the
correctly rounded one instead of the GPU's approximate one, which the Newton
step makes irrelevant), against the oracle's component-form equations and
against mpmath:
  - the table sine and cosine within 3.5e-16 relative over the rays' angles;
  - the seeded reciprocal within 2.5e-16 relative;
  - every derivative within 5e-14 of the size of the terms it is summed from
    (the largest derivative, and in Kerr the terms (u^2 + p_r^2) r / Sigma,
    u = P / Delta, that cancel in p_r' next to the horizon), r' and theta' in
    Kerr within 1e-13 relative, and 2H within 1e-14 of its terms.
Measured worst: 2.6e-16, 1.1e-16, 1.5e-14, 2.4e-14 and 2.8e-15."""
import subprocess

import numpy as np
import pytest

import oracle
from _df_host import build

HARNESS = r"""
#include "trace_device.cuh"
using namespace osiris_impl;
int main(int argc, char** argv) {
  trig_table_init();
  explog_table_init();
  const char op = argv[1][0];
  double in[10];  // 'e': kind, a or q, E, L, r, theta, p_r, p_theta; 's', 'r': x;
                  // 'k': integrator, a, E, L, r, theta, phi, p_r, p_theta, h
  const int n_in = op == 'e' ? 8 : op == 'k' ? 10 : 1;
  while (std::fread(in, sizeof(double), n_in, stdin) == (size_t)n_in) {
    if (op == 's') {
      double s, c;
      sincos_tab(in[0], s, c);
      const double out[2] = {s, c};
      std::fwrite(out, sizeof out, 1, stdout);
    } else if (op == 'r') {
      const double out = rcp64(in[0]);
      std::fwrite(&out, sizeof out, 1, stdout);
    } else if (op == 'k') {  // one Kerr attempt of the FP64 kernels' stepper
      RayK K;
      K.a = in[1];
      K.a2 = K.a * K.a;
      K.q = K.kap = 0.0;
      K.E = in[2];
      K.L = in[3];
      K.aE = K.a * K.E;
      K.aL = K.a * K.L;
      K.E2 = K.E + K.E;
      State y, o, d;
      y.r = in[4];
      y.th = in[5];
      y.ph = in[6];
      y.pr = in[7];
      y.pth = in[8];
      if (in[0] == 0.0) {
        double twoH;
        ck_step64<KerrMetric>(K, y, in[9], o, d, twoH);
      } else {
        Deriv k1, k7;
        rhs64_at<KerrMetric>(K, y, k1);
        dp_step64<KerrMetric>(K, y, in[9], k1, o, d, k7);
      }
      const double out[10] = {o.r, o.th, o.ph, o.pr, o.pth, d.r, d.th, d.ph, d.pr, d.pth};
      std::fwrite(out, sizeof out, 1, stdout);
    } else {
      RayK K;  // as the kernels' load_ray forms it
      K.a = in[0] == 0.0 ? in[1] : 0.0;
      K.a2 = K.a * K.a;
      K.q = in[0] == 0.0 ? 0.0 : in[1];
      K.kap = K.q * (2.0 + K.q);
      K.E = in[2];
      K.L = in[3];
      K.aE = K.a * K.E;
      K.aL = K.a * K.L;
      K.E2 = K.E + K.E;
      double dr, dth, dph, dpr, dpth, twoH, scale;
      if (in[0] == 0.0)
        rhs64(K, in[4], in[5], in[6], in[7], dr, dth, dph, dpr, dpth, twoH, scale);
      else
        rhs_q64(K, in[4], in[5], in[6], in[7], dr, dth, dph, dpr, dpth, twoH, scale);
      // the Kerr outputs carry a factor Sigma, returned as scale = 1 / Sigma
      const double out[6] = {dr * scale, dth * scale, dph * scale, dpr * scale, dpth * scale,
                             twoH};
      std::fwrite(out, sizeof out, 1, stdout);
    }
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def dev(tmp_path_factory):
    exe = build(tmp_path_factory, "rhs64", HARNESS, device_shims=True)

    def run(op, x, width):
        inp = np.ascontiguousarray(x, dtype=np.float64)
        p = subprocess.run([str(exe), op], input=inp.tobytes(), capture_output=True, check=True)
        return np.frombuffer(p.stdout, dtype=np.float64).reshape(-1, width)
    return run


def _mp():
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 120
    return mp


def test_table_sincos(dev):
    mp = _mp()
    rng = np.random.default_rng(1)
    th = np.concatenate([rng.uniform(-0.2, np.pi + 0.2, 4000),
                         rng.uniform(-1, 1, 500) * np.exp(rng.uniform(np.log(1e-12), 0, 500)),
                         np.pi + rng.uniform(-1, 1, 500) * np.exp(rng.uniform(np.log(1e-9), 0, 500))])
    out = dev("s", th, 2)
    worst = 0.0
    for t, (s, c) in zip(th, out):
        for got, want in ((s, mp.sin(mp.mpf(float(t)))), (c, mp.cos(mp.mpf(float(t))))):
            if abs(want) > 1e-300:
                worst = max(worst, float(abs(got - want) / abs(want)))
    assert worst <= 3.5e-16, worst


def test_seeded_reciprocal(dev):
    mp = _mp()
    rng = np.random.default_rng(2)
    x = np.exp(rng.uniform(-80.0, 80.0, 5000)) * rng.choice([-1.0, 1.0], 5000)
    out = dev("r", x, 1)[:, 0]
    worst = max(float(abs(mp.mpf(float(r)) * mp.mpf(float(v)) - 1)) for v, r in zip(x, out))
    assert worst <= 2.5e-16, worst


def _points(kind, params, n, seed, near_horizon=False):
    rng = np.random.default_rng(seed)
    rows = []
    for prm in params:
        r_h = 1.0 + np.sqrt(1.0 - prm * prm) if kind == 0 else 2.0
        for _ in range(n):
            r = (r_h * rng.uniform(1.02, 1.2) if near_horizon
                 else np.exp(rng.uniform(np.log(1.02 * r_h + 0.03), np.log(1000.0))))
            rows.append([kind, prm, 1.0, rng.uniform(-8.0, 8.0), r,
                         rng.uniform(0.05, np.pi - 0.05), 2.0 * rng.normal(), 5.0 * rng.normal()])
    return np.array(rows)


def _check(rows, out):
    for row, o in zip(rows, out):
        kind, prm, E, L, r, th, pr, pth = row
        sp = oracle.KERR if kind == 0 else oracle.QMETRIC
        kw = dict(a=prm) if kind == 0 else dict(q=prm)
        y6 = np.array([0.0, r, th, 0.0, pr, pth])
        dy = oracle.rhs_sp(sp, y6, E, L, **kw)
        scale = np.abs(dy[1:]).max()
        if kind == 0:
            delta = r * r - 2.0 * r + prm * prm
            sigma = r * r + prm * prm * np.cos(th) ** 2
            u = ((r * r + prm * prm) * E - prm * L) / delta
            scale += (u * u + pr * pr) * max(r, 1.0) / sigma
        err = np.abs(o[:5] - dy[1:])
        assert err.max() <= 5e-14 * scale, (row, o, dy)
        if kind == 0:
            assert err[0] <= 1e-13 * abs(dy[1]) and err[1] <= 1e-13 * abs(dy[2]), (row, o, dy)
        twoH = 2.0 * oracle.hamiltonian_sp(sp, y6, E, L, **kw)
        assert abs(o[5] - twoH) <= 1e-14 * scale * max(1.0, r), (row, o[5], twoH)


def test_kerr_rhs64_against_oracle(dev):
    rows = np.concatenate([_points(0, (0.0, 0.5, 0.9, 0.998), 250, 3),
                           _points(0, (0.998,), 300, 4, near_horizon=True)])
    _check(rows, dev("e", rows, 6))


def test_qmetric_rhs_q64_against_oracle(dev):
    rows = _points(1, (-0.5, 0.1, 0.5), 300, 5)
    _check(rows, dev("e", rows, 6))


def test_fp64_attempt_against_oracle_step(dev):
    """One Cash-Karp or Dormand-Prince attempt of the FP64 kernels (the
    derivatives' common factor 1/Sigma folded into the tableau coefficients)
    against the oracle's step: the fifth-order result within 2e-14 of
    1 + |y|, and the error norm, at the accept threshold of tol 1e-10,
    within 2e-5 of the oracle's (measured worst 2.9e-15 and 1.7e-6: the
    accept/reject decisions are the oracle's)."""
    rng = np.random.default_rng(6)
    rows = []
    for integ in (oracle.RKCK45, oracle.RKDP45):
        for a in (0.0, 0.5, 0.9, 0.998):
            r_h = 1.0 + np.sqrt(1.0 - a * a)
            for _ in range(200):
                r = np.exp(rng.uniform(np.log(1.1 * r_h), np.log(1000.0)))
                rows.append([integ, a, 1.0, rng.uniform(-6.0, 6.0), r,
                             rng.uniform(0.1, np.pi - 0.1), 0.3, -rng.uniform(0.0, 1.0),
                             3.0 * rng.normal(),
                             r * np.exp(rng.uniform(np.log(1e-4), np.log(0.05)))])
    rows = np.array(rows)
    out = dev("k", rows, 10)
    n_result = n_threshold = 0
    for row, o in zip(rows, out):
        integ, a, E, L, r, th, ph, pr, pth, h = row
        y6 = np.array([0.0, r, th, ph, pr, pth])
        y5, d = oracle.rk_step(int(integ), a, y6, E, L, h)
        scale = 1.0 + np.maximum(np.abs(y6[1:]), np.abs(y5[1:]))
        errn = np.max(np.abs(d[1:]) / scale)
        if errn <= 1e-9:
            n_result += 1
            assert np.max(np.abs(o[:5] - y5[1:]) / scale) <= 2e-14, (row, o[:5], y5)
        if 1e-10 <= errn <= 1e-9:
            n_threshold += 1
            assert abs(np.max(np.abs(o[5:]) / scale) / errn - 1.0) <= 2e-5, (row, o[5:], d)
    assert n_result > 800 and n_threshold >= 20

