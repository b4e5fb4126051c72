// Hamilton's equations in FP32 for the MIXED kernels: the separated form of
// rhs64 (trace_device.cuh, Sec. 2.1 on the metric of Sec. 4.3) with every
// operation in single precision, evaluated at the df64 stage input of the
// double-float stepper (step_df.cuh). Two quantities that FP32 would lose to
// cancellation are formed from both words of that input:
//   - Delta = (r - r+)(r - r-): the factor r - r+ vanishes at the horizon, so
//     it is taken as (r.hi - r+.hi) + (r.lo - r+.lo), whose leading difference
//     is exact there (Sterbenz); Delta keeps FP32 relative accuracy down to
//     the capture radius, where r^2 - 2r + a^2 in FP32 would keep none;
//   - the reduced angle t = theta - k pi/2 of sin and cos: k P1 is subtracted
//     from the leading word exactly (as in df_sincos), so sin theta keeps its
//     relative accuracy next to the poles.
// Every other operation has FP32 relative accuracy (~1e-7), the accuracy of
// the derivatives this returns. Like rhs_df it uses no CUDA built-in beyond
// the FP32 intrinsics, so it also compiles as host C++ for the CPU tests.
#pragma once

#include "df64.cuh"

namespace osiris_impl {

struct RayF32 {
  float a, a2, aE, aL, E, L, twoE;
  df rp;     // outer horizon radius r+ = 1 + sqrt(1 - a^2) (M = 1)
  float rm;  // inner horizon radius r- = 1 - sqrt(1 - a^2)
  float twoH0;
};

// sin and cos of a df64 angle in FP32: t = theta - k pi/2, |t| <= pi/4, then
// the Taylor polynomials of sin t (to t^9) and cos t (to t^10), whose
// truncation at |t| = pi/4 is below 3e-9 of the result.
__device__ __forceinline__ void sincos_f32(df th, float& s, float& c) {
  using namespace dfc;
  const float k = rintf(__fmul_rn(th.hi, 0.636619772367581343f));
  const float t = __fadd_rn(fmaf(-k, P1, th.hi), fmaf(-k, P2, th.lo));
  const float u = __fmul_rn(t, t);
  const float ps = fmaf(u, fmaf(u, fmaf(u, fmaf(u, I9H, -I7H), I5H), -I3H), 1.0f);
  const float st = __fmul_rn(t, ps);
  const float ct = fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, -I10, I8H), -I6H), I4H), -0.5f), 1.0f);
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

// The derivatives (r', theta', phi', p_r', p_theta') and 2 (H - H0) at
// (r, theta, p_r, p_theta), as rhs64 writes them, in FP32.
__device__ __forceinline__ void rhs_f32(const RayF32& K, df r, df th, df pr, df pth, float& dr,
                                        float& dth, float& dph, float& dpr, float& dpth,
                                        float& twoH) {
  float s, c;
  sincos_f32(th, s, c);
  const float rf = __fadd_rn(r.hi, r.lo);
  const float prf = __fadd_rn(pr.hi, pr.lo);
  const float ptf = __fadd_rn(pth.hi, pth.lo);
  const float dp = __fadd_rn(__fsub_rn(r.hi, K.rp.hi), __fsub_rn(r.lo, K.rp.lo));  // r - r+
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

}  // namespace osiris_impl
