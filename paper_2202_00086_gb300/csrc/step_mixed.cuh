// The embedded Runge-Kutta attempt of the MIXED kernels (Cash-Karp 4(5) and
// Dormand-Prince 5(4), Sec. 3.1) with FP32 stage derivatives: the state stays
// df64 and every stage input is that state plus an FP32 increment, handed to
// the FP32 evaluation unsummed (PointF32, rhs_f32.cuh) so that a point next
// to the horizon or a pole keeps what the evaluation needs of both words;
// the sums over stages - the increments of the stage inputs, the fifth-order
// increment and the error estimate - are FP32 sums of the FP32 derivatives.
//
// Precision. The derivatives k_s carry the FP32 rounding of the evaluation,
// a few units of 2^-24 |k|. Each FP32 sum over them adds one or two roundings
// of the same size relative to its result (|h sum a_ts k_s| <= ~|h k|), so the
// increment of a step keeps the error class of its derivatives; what FP32
// could not keep, the sum of a small increment and the state it is added to,
// is a df64 addition. The error estimate h sum_s (b_s - b*_s)(k_s - k_1) is
// summed from the differences e_s = k_s - k_1, each formed in FP32 with a
// rounding of 2^-24 |e_s| (much smaller than the rounding of k_s itself).
//
// The tableau is the one of step_df.cuh (kA, kCH, kBH, kDH) rounded to FP32.
// With e_s the stage inputs are y + h (c_t k_1 + sum_s a_ts e_s) and the
// fifth-order result y + h (k_1 + sum_s b_s e_s); both equal the usual forms
// since sum_s a_ts = c_t and sum_s b_s = 1. The stage loop is unrolled, so
// the tableau's entries are immediates and the stage selection costs nothing.
#pragma once

#include "df64.cuh"
#include "osiris.h"
#include "rhs_f32.cuh"
#include "step_df.cuh"

namespace osiris_impl {

// Dormand-Prince keeps k1 = f(y) between attempts (the seventh stage of the
// last accepted attempt), in FP32; Cash-Karp keeps nothing.
template <int INTEG>
struct LaneCacheF32 {
  __device__ __forceinline__ void reset() {}
  __device__ __forceinline__ void accepted() {}
};
template <>
struct LaneCacheF32<OSIRIS_RKDP45> {
  float k1[5], k7[5];
  float twoH1, twoH7;
  bool valid;
  __device__ __forceinline__ void reset() { valid = false; }
  __device__ __forceinline__ void accepted() {
#pragma unroll
    for (int c = 0; c < 5; ++c) k1[c] = k7[c];
    twoH1 = twoH7;
  }
};

// One attempt of length h.hi from y: o = fifth-order result (df64), d = fifth
// minus fourth order (FP32), twoH = 2 (H - H0) at y from the FP32 evaluation.
// Met::rhs_f evaluates Hamilton's equations in FP32 at a df64 point.
template <class Met, int INTEG>
__device__ __forceinline__ void rk_step_mixed(const typename Met::Ray& K,
                                              LaneCacheF32<INTEG>& LC, const StateDF& y, df h,
                                              StateDF& o, float d[5], float& twoH) {
  constexpr int I = (INTEG == OSIRIS_RKDP45) ? 1 : 0;
  constexpr int NS = (INTEG == OSIRIS_RKDP45) ? 7 : 6;
  const float hf = h.hi;
  float k1[5], sb[5], sd[5];
  float acc[4][4];  // sum_s a_ts e_s of stages t = 2..5; (r, theta, p_r, p_theta)
  bool need_k1 = true;
  twoH = 0.0f;
#pragma unroll
  for (int c = 0; c < 5; ++c) k1[c] = sb[c] = sd[c] = 0.0f;
  if constexpr (INTEG == OSIRIS_RKDP45) {
    need_k1 = !LC.valid;
    if (!need_k1) {
#pragma unroll
      for (int c = 0; c < 5; ++c) k1[c] = LC.k1[c];
      twoH = LC.twoH1;
    }
  }
#pragma unroll
  for (int t = 0; t < 4; ++t)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[t][c] = 0.0f;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    if (s == 0 && !need_k1) continue;
    PointF32 x;
    if (s == 0) {
      x.r = y.r;
      x.th = y.th;
      x.dr = x.dth = -0.0f;  // x + (-0) = x for every x
      x.pr = y.pr.hi;
      x.pth = y.pth.hi;
    } else if (INTEG == OSIRIS_RKDP45 && s == NS - 1) {
      // the fifth-order solution (first same as last)
      o.r = df_add_f(y.r, __fmul_rn(hf, __fadd_rn(k1[0], sb[0])));
      o.th = df_add_f(y.th, __fmul_rn(hf, __fadd_rn(k1[1], sb[1])));
      o.ph = df_add_f(y.ph, __fmul_rn(hf, __fadd_rn(k1[2], sb[2])));
      o.pr = df_add_f(y.pr, __fmul_rn(hf, __fadd_rn(k1[3], sb[3])));
      o.pth = df_add_f(y.pth, __fmul_rn(hf, __fadd_rn(k1[4], sb[4])));
      x.r = o.r;
      x.th = o.th;
      x.dr = x.dth = -0.0f;
      x.pr = o.pr.hi;
      x.pth = o.pth.hi;
    } else {
      const float cs = kCH[I][s];
      float inc[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int kc = c < 2 ? c : c + 1;  // skip phi in k
        const float fs = s >= 2 ? acc[s - 2][c] : 0.0f;
        inc[c] = __fmul_rn(hf, fmaf(cs, k1[kc], fs));
      }
      x.r = y.r;
      x.th = y.th;
      x.dr = inc[0];
      x.dth = inc[1];
      x.pr = __fadd_rn(y.pr.hi, inc[2]);
      x.pth = __fadd_rn(y.pth.hi, inc[3]);
    }
    float k[5], h2;
    Met::rhs_f(K, x, k[0], k[1], k[2], k[3], k[4], h2);
    if (s == 0) {
      twoH = h2;
#pragma unroll
      for (int c = 0; c < 5; ++c) k1[c] = k[c];
      continue;
    }
    if constexpr (INTEG == OSIRIS_RKDP45) {
      if (s == NS - 1) {
#pragma unroll
        for (int c = 0; c < 5; ++c) LC.k7[c] = k[c];
        LC.twoH7 = h2;
      }
    }
    float e[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) e[c] = __fsub_rn(k[c], k1[c]);
    const float ds[4] = {e[0], e[1], e[3], e[4]};
#pragma unroll
    for (int t = 2; t < 6; ++t) {
      if (t > s) {
        const float a = kA[I][t][s];
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[t - 2][c] = fmaf(a, ds[c], acc[t - 2][c]);
      }
    }
    if (s >= 2) {
      const float bw = kBH[I][s];
      const float dw = kDH[I][s];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        sb[c] = fmaf(bw, e[c], sb[c]);
        sd[c] = fmaf(dw, e[c], sd[c]);
      }
    }
  }
  if constexpr (INTEG == OSIRIS_RKDP45) {
    LC.valid = true;
#pragma unroll
    for (int c = 0; c < 5; ++c) LC.k1[c] = k1[c];  // unchanged when the attempt is rejected
    LC.twoH1 = twoH;
  } else {
    o.r = df_add_f(y.r, __fmul_rn(hf, __fadd_rn(k1[0], sb[0])));
    o.th = df_add_f(y.th, __fmul_rn(hf, __fadd_rn(k1[1], sb[1])));
    o.ph = df_add_f(y.ph, __fmul_rn(hf, __fadd_rn(k1[2], sb[2])));
    o.pr = df_add_f(y.pr, __fmul_rn(hf, __fadd_rn(k1[3], sb[3])));
    o.pth = df_add_f(y.pth, __fmul_rn(hf, __fadd_rn(k1[4], sb[4])));
  }
#pragma unroll
  for (int c = 0; c < 5; ++c) d[c] = __fmul_rn(hf, sd[c]);
}

}  // namespace osiris_impl
