// The double-float embedded Runge-Kutta attempt of the DF64 kernels
// (Cash-Karp 4(5) and Dormand-Prince 5(4), Sec. 3.1): the df64 state, the
// tableaus as float pairs, the per-lane stage cache and rk_step_df. It uses
// only df64 arithmetic and a metric policy for the evaluation, so it also
// compiles as host C++, which is how one attempt is compared with the
// oracle's step on the CPU.
#pragma once

#include "df64.cuh"
#include "osiris.h"

#ifdef __CUDACC__
#define OSIRIS_DF_TABLEAU static __constant__
#else
#define OSIRIS_DF_TABLEAU static const
#endif

namespace osiris_impl {

struct StateDF {
  df r, th, ph, pr, pth;
};

// Tableaus for the df64 stepper, [integrator][stage]; stage s = 0..6 is the
// tableau's stage s + 1. kA[i][t][s] = a_{t+1, s+1} in FP32 (the O(h) parts of
// stage inputs); c_s and b_s as df, b_s - b*_s in FP32.
OSIRIS_DF_TABLEAU float kA[2][7][7] = {
    {{0, 0, 0, 0, 0, 0, 0},
     {0, 0, 0, 0, 0, 0, 0},
     {0, 9.0f / 40.0f, 0, 0, 0, 0, 0},
     {0, -9.0f / 10.0f, 6.0f / 5.0f, 0, 0, 0, 0},
     {0, 5.0f / 2.0f, -70.0f / 27.0f, 35.0f / 27.0f, 0, 0, 0},
     {0, 175.0f / 512.0f, 575.0f / 13824.0f, 44275.0f / 110592.0f, 253.0f / 4096.0f, 0, 0},
     {0, 0, 0, 0, 0, 0, 0}},
    {{0, 0, 0, 0, 0, 0, 0},
     {0, 0, 0, 0, 0, 0, 0},
     {0, 9.0f / 40.0f, 0, 0, 0, 0, 0},
     {0, -56.0f / 15.0f, 32.0f / 9.0f, 0, 0, 0, 0},
     {0, -25360.0f / 2187.0f, 64448.0f / 6561.0f, -212.0f / 729.0f, 0, 0, 0},
     {0, -355.0f / 33.0f, 46732.0f / 5247.0f, 49.0f / 176.0f, -5103.0f / 18656.0f, 0, 0},
     {0, 0, 0, 0, 0, 0, 0}}};
OSIRIS_DF_TABLEAU float kCH[2][7] = {
    {0.0f, 0.20000000298023224f, 0.30000001192092896f, 0.6000000238418579f, 1.0f, 0.875f, 0.0f},
    {0.0f, 0.20000000298023224f, 0.30000001192092896f, 0.800000011920929f, 0.8888888955116272f,
     1.0f, 1.0f}};
OSIRIS_DF_TABLEAU float kCL[2][7] = {
    {0.0f, -2.9802322831784522e-09f, -1.1920929132713809e-08f, -2.3841858265427618e-08f, 0.0f,
     0.0f, 0.0f},
    {0.0f, -2.9802322831784522e-09f, -1.1920929132713809e-08f, -1.1920929132713809e-08f,
     -6.622738357719982e-09f, 0.0f, 0.0f}};
// fifth-order weights b_s for s >= 2 (b_1 multiplies d_1 = 0; b_2 = 0 in both)
OSIRIS_DF_TABLEAU float kBH[2][7] = {
    {0.0f, 0.0f, 0.4025764763355255f, 0.21043771505355835f, 0.0f, 0.2891021966934204f, 0.0f},
    {0.0f, 0.0f, 0.44923630356788635f, 0.6510416865348816f, -0.32237619161605835f,
     0.130952388048172f, 0.0f}};
OSIRIS_DF_TABLEAU float kBL[2][7] = {
    {0.0f, 0.0f, 1.3197485770888306e-08f, -4.615847704059206e-09f, 0.0f, 5.452259976834739e-09f,
     0.0f},
    {0.0f, 0.0f, -5.2749844492439024e-09f, -1.9868215517249155e-08f, 1.2370775515080368e-08f,
     -7.095791065836465e-09f, 0.0f}};
// b_s - b*_s for s >= 2 (zero for s = 1 in both), in FP32 (the error sum is
// an FP32 sum, see rk_step_df)
OSIRIS_DF_TABLEAU float kDH[2][7] = {
    {0.0f, 0.0f, 0.018668586388230324f, -0.03415502607822418f, -0.01932198740541935f,
     0.03910220041871071f, 0.0f},
    {0.0f, 0.0f, -0.004252770449966192f, 0.03697916492819786f, -0.05086379870772362f,
     0.041904762387275696f, -0.02500000037252903f}};

struct DerivDF {
  df r, th, ph, pr, pth;
  float twoH;
};

// Stage values carried between attempts: Dormand-Prince keeps k1 = f(y) (the
// seventh stage of the last accepted attempt); Cash-Karp keeps nothing.
template <int INTEG>
struct LaneCacheDF {
  __device__ __forceinline__ void reset() {}
  __device__ __forceinline__ void accepted() {}
};
template <>
struct LaneCacheDF<OSIRIS_RKDP45> {
  DerivDF k1, k7;
  bool valid;
  __device__ __forceinline__ void reset() { valid = false; }
  __device__ __forceinline__ void accepted() { k1 = k7; }
};

// One embedded Runge-Kutta attempt of length h from y, all in df64: o =
// fifth-order result, d = fifth minus fourth order. The stages share one copy
// of the equations; as soon as stage s gives d_s = k_s - k_1 it is folded
// into the FP32 sums of the later stage inputs, the df64 increment sum and
// the FP32 error sum, so no stage value is kept in memory.
//
// The error sum h sum_s (b_s - b*_s) d_s cancels from terms of size
// T ~ h |d_s| / 30 to the local error D ~ tol |y|. Each d_s is exact to
// df64 precision (k_s and k_1 are df64 values), so summing its leading word
// in FP32 costs only the FP32 rounding of the terms, ~2^-24 T; with
// |d_s| ~ (h / tau) |k| and D ~ (h / tau)^5 |y| (tau: time scale of the
// solution, |y| ~ tau |k|) that is a relative error of ~2^-24 (h / tau)^-3 / 30
// in D: about 0.2 % at tol = 1e-10 and 3 % at 1e-12, inside the
// controller's safety factor. (An FP32 evaluation of the equations, by
// contrast, would put the rounding of k itself, 2^-24 |k|, into every d_s.)
//
// Dormand-Prince: the seventh stage input is the fifth-order solution itself
// (formed in df64 exactly as o), its derivative is cached as the next k1, and
// k1 is evaluated here only when the cache is empty. twoH is 2 (H - H0) at y.
template <class Met, int INTEG>
__device__ __forceinline__ void rk_step_df(const typename Met::Ray& K, LaneCacheDF<INTEG>& LC,
                                           const StateDF& y, df h, StateDF& o, float d[5],
                                           float& twoH) {
  constexpr int I = (INTEG == OSIRIS_RKDP45) ? 1 : 0;
  constexpr int NS = (INTEG == OSIRIS_RKDP45) ? 7 : 6;
  df k1[5], hk1[5], sb[5];
  float sd[5];
  float acc[4][4];  // FP32 sums sum_j a_tj d_j of stages t = 2..5; (r, theta, p_r, p_theta)
  bool need_k1 = true;
  twoH = 0.0f;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    k1[c] = hk1[c] = sb[c] = mk(0.0f, 0.0f);
    sd[c] = 0.0f;
  }
  if constexpr (INTEG == OSIRIS_RKDP45) {
    need_k1 = !LC.valid;
    if (!need_k1) {
      k1[0] = LC.k1.r;
      k1[1] = LC.k1.th;
      k1[2] = LC.k1.ph;
      k1[3] = LC.k1.pr;
      k1[4] = LC.k1.pth;
      twoH = LC.k1.twoH;
#pragma unroll
      for (int c = 0; c < 5; ++c) hk1[c] = df_mul(h, k1[c]);
    }
  }
#pragma unroll
  for (int t = 0; t < 4; ++t)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[t][c] = 0.0f;
  const df y4[4] = {y.r, y.th, y.pr, y.pth};
  const float hf = h.hi;
  // The stage loop stays rolled: unrolled, the six inlined double-float
  // evaluations overflow the instruction cache (Kerr set at tol 1e-10: 20.1
  // Mrays/s rolled, 14.3 unrolled), unlike the MIXED stepper's FP32 ones.
#pragma unroll 1
  for (int s = 0; s < NS; ++s) {
    if (s == 0 && !need_k1) continue;
    df in[4];
    if (s == 0) {
#pragma unroll
      for (int c = 0; c < 4; ++c) in[c] = y4[c];
    } else if (INTEG == OSIRIS_RKDP45 && s == NS - 1) {
      // the fifth-order solution (first same as last)
      o.r = df_add(y.r, df_mul(h, df_add_u(k1[0], sb[0])));
      o.th = df_add(y.th, df_mul(h, df_add_u(k1[1], sb[1])));
      o.ph = df_add(y.ph, df_mul(h, df_add_u(k1[2], sb[2])));
      o.pr = df_add(y.pr, df_mul(h, df_add_u(k1[3], sb[3])));
      o.pth = df_add(y.pth, df_mul(h, df_add_u(k1[4], sb[4])));
      in[0] = o.r;
      in[1] = o.th;
      in[2] = o.pr;
      in[3] = o.pth;
    } else {
      const df cs = mk(kCH[I][s], kCL[I][s]);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int kc = c < 2 ? c : c + 1;  // skip phi in k
        const float fs = s == 2 ? acc[0][c] : s == 3 ? acc[1][c] : s == 4 ? acc[2][c]
                       : s == 5 ? acc[3][c] : 0.0f;
        in[c] = df_add_f_u(df_add_u(y4[c], df_mul(hk1[kc], cs)), __fmul_rn(hf, fs));
      }
    }
    df k[5];
    float h2;
    Met::rhs(K, in[0], in[1], in[2], in[3], k[0], k[1], k[2], k[3], k[4], h2);
    if (s == 0) {
      twoH = h2;
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        k1[c] = k[c];
        hk1[c] = df_mul(h, k[c]);
      }
      continue;
    }
    if constexpr (INTEG == OSIRIS_RKDP45) {
      if (s == NS - 1) {
        LC.k7.r = k[0];
        LC.k7.th = k[1];
        LC.k7.ph = k[2];
        LC.k7.pr = k[3];
        LC.k7.pth = k[4];
        LC.k7.twoH = h2;
      }
    }
    df e[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) e[c] = df_sub(k[c], k1[c]);  // renormalised: the error sum cancels to O(h^5)
    const float ds[4] = {e[0].hi, e[1].hi, e[3].hi, e[4].hi};
#pragma unroll
    for (int t = 2; t < 6; ++t) {
      if (t > s) {
        const float a = kA[I][t][s];
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[t - 2][c] = fmaf(a, ds[c], acc[t - 2][c]);
      }
    }
    if (s >= 2) {
      const df bw = mk(kBH[I][s], kBL[I][s]);
      const float dw = kDH[I][s];
      const bool has_b = (bw.hi != 0.0f);
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        if (has_b) sb[c] = df_add_u(sb[c], df_mul(e[c], bw));
        sd[c] = fmaf(dw, e[c].hi, sd[c]);
      }
    }
  }
  if constexpr (INTEG == OSIRIS_RKDP45) {
    LC.valid = true;
    LC.k1.r = k1[0];  // k1 of this attempt's start (unchanged when the attempt is rejected)
    LC.k1.th = k1[1];
    LC.k1.ph = k1[2];
    LC.k1.pr = k1[3];
    LC.k1.pth = k1[4];
    LC.k1.twoH = twoH;
  } else {
    o.r = df_add(y.r, df_mul(h, df_add_u(k1[0], sb[0])));
    o.th = df_add(y.th, df_mul(h, df_add_u(k1[1], sb[1])));
    o.ph = df_add(y.ph, df_mul(h, df_add_u(k1[2], sb[2])));
    o.pr = df_add(y.pr, df_mul(h, df_add_u(k1[3], sb[3])));
    o.pth = df_add(y.pth, df_mul(h, df_add_u(k1[4], sb[4])));
  }
#pragma unroll
  for (int c = 0; c < 5; ++c) d[c] = __fmul_rn(h.hi, sd[c]);
}

}  // namespace osiris_impl

#undef OSIRIS_DF_TABLEAU
