"""The double-float evaluations of Hamilton's equations used by the DF64
kernels (rhs_df.cuh: Kerr in the separated form, the q-metric in the
collected form), compiled as host C++, against the oracle's component-form
equations at random phase-space points, off the constraint surface and down
to 1.02 horizon radii.

Double-float carries 48 significand bits. Each derivative must agree with the
oracle to 3e-11 of the size of the terms it is summed from: the largest
derivative at that point, and in Kerr also (u^2 + p_r^2) r / Sigma with
u = P / Delta, the terms that cancel in p_r' next to the horizon (measured
worst: 9e-12 there, 1.6e-12 elsewhere, 1.3e-13 in the q-metric). r' and
theta' (no cancellation: Delta p_r / Sigma and p_theta / Sigma in Kerr) must
agree to 1e-11 relative. The reported 2 (H - H0) is an FP32 word (it only has
to resolve the deviation on the mass shell), so it is held to FP32 precision
of |2H|. A reciprocal taken of an unrenormalised Delta next to the horizon
once left 3e-10 errors in every Kerr derivative; these bounds catch that."""
import subprocess

import numpy as np
import pytest

import oracle
from _df_host import build

HARNESS = r"""
#include <cstdlib>
#include "rhs_df.cuh"
using namespace osiris_impl;
static double d(df x) { return (double)x.hi + (double)x.lo; }
// x as an unrenormalised pair whose low word is k ulp(hi) away from the
// renormalised one (hi moved by -k ulp, lo by +k ulp): the stage inputs of the
// DF64 kernels reach the evaluation in this form.
static df skew(double x, int k) {
  df v = df_from_double(x);
  if (k == 0 || v.hi == 0.0f) return v;
  const float h = nextafterf(v.hi, k > 0 ? -INFINITY : INFINITY);
  const float h2 = k > 1 ? nextafterf(h, k > 0 ? -INFINITY : INFINITY) : h;
  return mk(h2, (float)(x - (double)h2));
}
int main(int argc, char** argv) {
  const int k = argc > 1 ? atoi(argv[1]) : 0;
  double in[9];  // kind (0 Kerr, 1 q-metric), a or q, E, L, H0, r, theta, p_r, p_theta
  while (std::fread(in, sizeof in, 1, stdin) == 1) {
    const double E = in[2], L = in[3], H0 = in[4];
    const df r = skew(in[5], k), th = skew(in[6], k);
    const df pr = skew(in[7], k), pth = skew(in[8], k);
    df dr, dth, dph, dpr, dpth;
    float twoH;
    if (in[0] == 0.0) {  // ray constants formed as the DF64 kernels form them
      const double a = in[1];
      RayDF k;
      k.a = df_from_double(a);
      k.a2 = df_from_double(a * a);
      k.aE = df_from_double(a * E);
      k.aL = df_from_double(a * L);
      k.E = df_from_double(E);
      k.L = df_from_double(L);
      k.twoE = df_scale(k.E, 2.0f);
      k.twoH0 = (float)(2.0 * H0);
      rhs_df(k, r, th, pr, pth, dr, dth, dph, dpr, dpth, twoH);
    } else {
      const double q = in[1];
      RayQDF k;
      k.E = df_from_double(E);
      k.L = df_from_double(L);
      k.q = df_from_double(q);
      k.kap = df_from_double(q * (2.0 + q));
      k.nq1 = df_from_double(-(1.0 + q));
      k.E2 = df_from_double(E * E);
      k.twoH0 = (float)(2.0 * H0);
      rhs_q_df(k, r, th, pr, pth, dr, dth, dph, dpr, dpth, twoH);
    }
    const double out[6] = {d(dr), d(dth), d(dph), d(dpr), d(dpth), (double)twoH};
    std::fwrite(out, sizeof out, 1, stdout);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def rhs_df(tmp_path_factory):
    exe = build(tmp_path_factory, "rhs_df", HARNESS)

    def run(rows, skew=0):
        inp = np.ascontiguousarray(rows, dtype=np.float64)
        p = subprocess.run([str(exe), str(skew)], input=inp.tobytes(), capture_output=True,
                           check=True)
        return np.frombuffer(p.stdout, dtype=np.float64).reshape(-1, 6)
    return run


def _points(kind, params, n, seed):
    rng = np.random.default_rng(seed)
    rows = []
    for prm in params:
        r_min = 1.02 * (1.0 + np.sqrt(1.0 - prm * prm)) if kind == 0 else 2.05
        for _ in range(n):
            rows.append([kind, prm, 1.0, rng.uniform(-8.0, 8.0), 0.0,
                         np.exp(rng.uniform(np.log(r_min), np.log(1000.0))),
                         rng.uniform(0.05, np.pi - 0.05), 2.0 * rng.normal(), 5.0 * rng.normal()])
    return np.array(rows)


def _check(rows, out):
    for row, o in zip(rows, out):
        kind, prm, E, L, H0, r, th, pr, pth = row
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
        assert err.max() <= 3e-11 * scale, (row, o, dy)
        if kind == 0:
            assert err[0] <= 1e-11 * abs(dy[1]) and err[1] <= 1e-11 * abs(dy[2]), (row, o, dy)
        twoH = 2.0 * (oracle.hamiltonian_sp(sp, y6, E, L, **kw) - H0)
        assert abs(o[5] - twoH) <= 2.4e-7 * abs(twoH) + 1e-12, (row, o[5], twoH)


def test_kerr_rhs_df_against_oracle(rhs_df):
    rows = _points(0, (0.0, 0.5, 0.9, 0.998), 250, 3)
    _check(rows, rhs_df(rows))


def test_kerr_rhs_df_next_to_the_horizon(rhs_df):
    """r within 1.02..1.2 horizon radii at a = 0.998, where Delta cancels."""
    rows = _points(0, (0.998,), 300, 4)
    r_h = 1.0 + np.sqrt(1.0 - 0.998 ** 2)
    rows[:, 5] = r_h * np.random.default_rng(5).uniform(1.02, 1.2, len(rows))
    _check(rows, rhs_df(rows))


def test_qmetric_rhs_df_against_oracle(rhs_df):
    rows = _points(1, (-0.5, 0.1, 0.5), 250, 6)
    _check(rows, rhs_df(rows))


def test_massive_particle_shell(rhs_df):
    """H0 = -1/2: the reported deviation 2 (H - H0) is formed from the
    double-float 2H, so it resolves |H - H0| on the shell."""
    rows = _points(0, (0.9,), 50, 7)
    rows[:, 4] = -0.5
    _check(rows, rhs_df(rows))
    rows = _points(1, (0.3,), 50, 8)
    rows[:, 4] = -0.5
    _check(rows, rhs_df(rows))


def test_unrenormalised_inputs(rhs_df):
    """Inputs whose low word is two ulp of the high word off the renormalised
    pair (the form in which the kernels' stage inputs arrive) give the same
    accuracy, next to the horizon included."""
    rows = np.concatenate([_points(0, (0.5, 0.998), 150, 9), _points(1, (-0.5, 0.5), 150, 10)])
    r_h = 1.0 + np.sqrt(1.0 - 0.998 ** 2)
    near = rows[:, 1] == 0.998
    rows[near, 5] = r_h * np.random.default_rng(11).uniform(1.02, 1.2, int(near.sum()))
    _check(rows, rhs_df(rows, skew=2))
