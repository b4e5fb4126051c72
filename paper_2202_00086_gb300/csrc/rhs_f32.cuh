// Hamilton's equations in FP32 for the MIXED kernels: the separated form of
// rhs64 (trace_device.cuh, Sec. 2.1 on the metric of Sec. 4.3) with every
// operation in single precision, evaluated at a stage input of the MIXED
// stepper (step_mixed.cuh). A stage input is the df64 state plus an FP32
// increment; r and theta are passed in that form (PointF32), because two
// quantities that FP32 would lose to cancellation are formed from the base's
// two words and the increment without rounding the sum first:
//   - Delta = (r - r+)(r - r-): the factor r - r+ vanishes at the horizon, so
//     it is taken as ((r.hi - r+.hi) + dr) + (r.lo - r+.lo), whose leading
//     difference is exact there (Sterbenz); Delta keeps FP32 relative
//     accuracy down to the capture radius, where r^2 - 2r + a^2 in FP32 would
//     keep none;
//   - the reduced angle t = theta - k pi/2 of sin and cos: k P1 is subtracted
//     from the base's leading word exactly (as in df_sincos) before the
//     increment is added, so sin theta keeps its relative accuracy next to
//     the poles.
// p_r and p_theta enter only as FP32 values. Every other operation has FP32
// relative accuracy (~1e-7), the accuracy of the derivatives this returns.
// The q-metric evaluation (rhs_q_f32, Appendix A) does the same with r - 2,
// the factor of f = 1 - 2/r that vanishes at its inner surface, and takes the
// powers f^q and X^k from the FP32 exp and log intrinsics. Like rhs_df it uses
// no CUDA built-in beyond the FP32 intrinsics, so it also compiles as host
// C++ for the CPU tests.
#pragma once

#include "df64.cuh"

namespace osiris_impl {

// The point of an evaluation: r = r.hi + r.lo + dr and theta = th.hi + th.lo
// + dth (a df64 base and an FP32 increment, dr = dth = -0 for the base
// itself), p_r and p_theta in FP32.
struct PointF32 {
  df r, th;
  float dr, dth, pr, pth;
};

struct RayF32 {
  float a, a2, aE, aL, E, L, twoE;
  df rp;     // outer horizon radius r+ = 1 + sqrt(1 - a^2) (M = 1)
  float rm;  // inner horizon radius r- = 1 - sqrt(1 - a^2)
  float twoH0;
};

// sin and cos of th + dth (a df64 base and an FP32 increment) in FP32:
// t = theta - k pi/2, |t| <= pi/4 (k from the rounded sum; th.hi - k P1 is
// exact, Sterbenz), then the Taylor polynomials of sin t (to t^9) and cos t
// (to t^10), whose truncation at |t| = pi/4 is below 3e-9 of the result.
__device__ __forceinline__ void sincos_f32(df th, float dth, float& s, float& c) {
  using namespace dfc;
  const float k = rintf(__fmul_rn(__fadd_rn(th.hi, dth), 0.636619772367581343f));
  const float t = __fadd_rn(__fadd_rn(fmaf(-k, P1, th.hi), dth), fmaf(-k, P2, th.lo));
  const float u = __fmul_rn(t, t);
  const float ps = fmaf(u, fmaf(u, fmaf(u, fmaf(u, I9H, -I7H), I5H), -I3H), 1.0f);
  const float st = __fmul_rn(t, ps);
  const float ct =
      fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, -I10, I8H), -I6H), I4H), -0.5f), 1.0f);
  const int q = ((int)k) & 3;
  if (q == 0) {
    s = st;
    c = ct;
  } else if (q == 1) {
    s = ct;
    c = -st;
  } else if (q == 2) {
    s = -st;
    c = -ct;
  } else {
    s = -ct;
    c = st;
  }
}

// The derivatives (r', theta', phi', p_r', p_theta') and 2 (H - H0) at x,
// as rhs64 writes them, in FP32.
__device__ __forceinline__ void rhs_f32(const RayF32& K, const PointF32& x, float& dr,
                                        float& dth, float& dph, float& dpr, float& dpth,
                                        float& twoH) {
  float s, c;
  sincos_f32(x.th, x.dth, s, c);
  const float rf = __fadd_rn(x.r.hi, x.dr);
  const float prf = x.pr;
  const float ptf = x.pth;
  // r - r+ (the differences of the words are exact next to the horizon)
  const float dp = __fadd_rn(__fadd_rn(__fsub_rn(x.r.hi, K.rp.hi), x.dr),
                             __fsub_rn(x.r.lo, K.rp.lo));
  const float Delta = __fmul_rn(dp, __fsub_rn(rf, K.rm));
  const float ra2 = fmaf(rf, rf, K.a2);  // r^2 + a^2
  const float a2s = __fmul_rn(K.a2, s);
  const float Sigma = fmaf(-a2s, s, ra2);  // r^2 + a^2 cos^2 (r > a: no cancellation)
  const float P = fmaf(ra2, K.E, -K.aL);
  const float DS = __fmul_rn(Delta, Sigma);
  // one reciprocal of Delta Sigma sin gives 1/Sigma, 1/Delta and 1/sin
  const float inv = __fdividef(1.0f, __fmul_rn(DS, s));
  const float sinv = __fmul_rn(s, inv);  // 1 / (Delta Sigma)
  const float iSig = __fmul_rn(Delta, sinv);
  const float iDel = __fmul_rn(Sigma, sinv);
  const float is = __fmul_rn(DS, inv);
  const float Lis = __fmul_rn(K.L, is);  // L / sin
  const float W = fmaf(-K.aE, s, Lis);
  const float u = __fmul_rn(P, iDel);
  const float Dpr = __fmul_rn(Delta, prf);
  const float N = fmaf(Dpr, prf, fmaf(ptf, ptf, fmaf(W, W, -__fmul_rn(P, u))));
  const float NiS = __fmul_rn(N, iSig);
  dr = __fmul_rn(Dpr, iSig);
  dth = __fmul_rn(ptf, iSig);
  dph = __fmul_rn(fmaf(W, is, __fmul_rn(K.a, u)), iSig);
  // p_r' Sigma = Y + r (X - Y), Y = u^2 + p_r^2, X = 2H + 2 E u
  const float Y = fmaf(u, u, __fmul_rn(prf, prf));
  const float X = fmaf(K.twoE, u, NiS);
  dpr = __fmul_rn(iSig, fmaf(rf, __fsub_rn(X, Y), Y));
  dpth = __fmul_rn(__fmul_rn(c, iSig), fmaf(W, fmaf(Lis, is, K.aE), -__fmul_rn(a2s, NiS)));
  twoH = __fsub_rn(NiS, K.twoH0);
}

struct RayQF32 {
  float E, L, q, kap, nq1, E2;  // kap = q (2 + q), nq1 = -(1 + q), E2 = E^2
  float twoH0;
};

// The q-metric (Appendix A) in FP32: the collected form of rhs_q_df
// (rhs_df.cuh) and rhs_q64, the derivatives from the four terms of 2H and
// their logarithmic derivatives, with f = (r - 2) / r and X = 1 + sin^2 / D,
// D = r (r - 2).
__device__ __forceinline__ void rhs_q_f32(const RayQF32& K, const PointF32& x, float& dr,
                                          float& dth, float& dph, float& dpr, float& dpth,
                                          float& twoH) {
  float s, c;
  sincos_f32(x.th, x.dth, s, c);
  const float rf = __fadd_rn(x.r.hi, x.dr);
  const float prf = x.pr;
  const float ptf = x.pth;
  // r - 2, exact next to r = 2
  const float rm2 = __fadd_rn(__fadd_rn(__fsub_rn(x.r.hi, 2.0f), x.dr), x.r.lo);
  const float iD = __fdividef(1.0f, __fmul_rn(rf, rm2));
  const float ir = __fmul_rn(rm2, iD);  // 1/r
  const float f = __fmul_rn(rm2, ir);   // 1 - 2/r
  const float s2 = __fmul_rn(s, s);
  const float is2 = __fdividef(1.0f, s2);
  const float X = fmaf(s2, iD, 1.0f);
  const float iX = __fdividef(1.0f, X);
  const float fq = __expf(__fmul_rn(K.q, __logf(f)));
  const float fXk = __fmul_rn(fq, __expf(__fmul_rn(K.kap, __logf(X))));
  const float ir2 = __fmul_rn(ir, ir);
  const float gtt = -__fdividef(1.0f, __fmul_rn(f, fq));
  dr = __fmul_rn(__fmul_rn(f, fXk), prf);
  dth = __fmul_rn(__fmul_rn(fXk, ir2), ptf);
  dph = __fmul_rn(__fmul_rn(__fmul_rn(fq, ir2), is2), K.L);
  // the four terms of 2H and their logarithmic derivatives
  const float Ht = __fmul_rn(gtt, K.E2);
  const float Hr = __fmul_rn(dr, prf), Hth = __fmul_rn(dth, ptf), Hph = __fmul_rn(dph, K.L);
  twoH = __fsub_rn(__fadd_rn(__fadd_rn(Ht, Hr), __fadd_rn(Hth, Hph)), K.twoH0);
  const float iDX = __fmul_rn(iD, iX);
  const float a1 = __fmul_rn(K.nq1, iD);
  const float a2 = __fmul_rn(__fmul_rn(__fmul_rn(K.kap, s2), __fsub_rn(rf, 1.0f)),
                             __fmul_rn(iD, iDX));
  const float a3 = fmaf(-K.q, iD, ir);
  const float HrHth = __fadd_rn(Hr, Hth);
  dpr = fmaf(a1, __fsub_rn(Hr, Ht), fmaf(a2, HrHth, __fmul_rn(a3, __fadd_rn(Hth, Hph))));
  dpth = __fmul_rn(__fmul_rn(c, s),
                   fmaf(-__fmul_rn(K.kap, iDX), HrHth, __fmul_rn(Hph, is2)));
}

}  // namespace osiris_impl
