// exp and log of double-float (df64) values, for the q-metric's powers f^q and
// X^k (Appendix A) in the double-float kernels. The reductions are those of
// the double-precision pair in explog.cuh (Tang's table-driven methods, ACM
// TOMS 1989 and 1990), carried out in df64 with float-pair tables:
//   exp: y = (64 m + j) ln2/64 + r, |r| <= ln2/128; ln2/64 split into three
//        floats (the first of 9 bits, so n times it and its difference from
//        y are exact); exp(r) - 1 = r + r^2 (1/2 + r (1/6 + r/24 + r^2/120)),
//        the terms below 2^-48 of the result in FP32.
//   log: x = 2^k m, F = 1 + j/128 nearest m (F >= 1.5 stored as F/2 with
//        k + 1), u = (m - F)/F with m - F exact; log1p(u) through u^7, the
//        terms below 2^-48 in FP32; k ln2 with ln2 split into three floats
//        (the first of 15 bits, so k times it is exact).
// Both stay within 4 units of 2^-48 relative of the exact value (measured
// worst cases 1.6 for exp, 2.4 for log) for -69 < y < 80 and x in
// [2^-100, 2^100]. Below y = -69 the low word of the result is subnormal and
// the relative precision falls towards 2^-35 at y = -80; for |y| >= 80, x
// outside that range, or NaN, they return the FP32 library value. A ray
// outside the capture radius never produces such arguments. The functions
// compile as host C++ as well (the tables are plain arrays there), which is
// how their error bound is tested.
#pragma once

#include "df64.cuh"
#include "explog_tables.h"

namespace osiris_impl {

struct alignas(8) ExpEntryDF {  // 2^(j/64) = hi + lo
  float hi, lo;
};

struct alignas(16) LogEntryDF {
  df logF;  // log F_j, or log(F_j / 2) for j >= 64
  df rcpF;  // 1 / F_j
};

#ifdef __CUDACC__
#define OSIRIS_EXPLOG_DF_STORAGE static __device__ const
#else
#define OSIRIS_EXPLOG_DF_STORAGE static const
#endif
OSIRIS_EXPLOG_DF_STORAGE ExpEntryDF kT2DF[64] = {OSIRIS_EXPLOG_T2_DF};
OSIRIS_EXPLOG_DF_STORAGE LogEntryDF kLgDF[129] = {OSIRIS_EXPLOG_LG_DF};
#undef OSIRIS_EXPLOG_DF_STORAGE

namespace dfe {
constexpr float IL = 0x1.715476p+6f;       // 64 / ln2
constexpr float L1 = 0x1.63p-7f;           // ln2/64 = L1 + L2 + L3 (+ 2e-22)
constexpr float L2 = -0x1.bd0106p-19f;
constexpr float L3 = 0x1.cf79acp-46f;
constexpr float LN1 = 0x1.62e4p-1f;        // ln2 = LN1 + LN2 + LN3 (+ 1e-21)
constexpr float LN2 = 0x1.7f7d1cp-20f;
constexpr float LN3 = 0x1.ef357ap-45f;
constexpr float T3H = 0x1.555556p-2f;      // 1/3 = T3H + T3L
constexpr float T3L = -0x1.555556p-27f;
constexpr float I3H = 0.1666666716337204f;  // 1/6 = I3H + I3L
constexpr float I3L = -4.967053879312289e-09f;
}  // namespace dfe

__device__ __forceinline__ df df_exp(df y) {
  using namespace dfe;
  if (!(fabsf(y.hi) < 80.0f)) return mk(expf(y.hi), 0.0f);
  const float n = rintf(__fmul_rn(y.hi, IL));  // |n| < 2^13
  const int ni = (int)n;
  // r = y - n ln2/64: y.hi - n L1 is exact, then the two smaller parts
  const float t = fmaf(-n, L1, y.hi);
  const df nl = two_prod(n, L2);
  const df r = df_sub(two_sum(t, y.lo), mk(nl.hi, fmaf(n, L3, nl.lo)));
  // |r| <= ln2/128: each sum below adds a term smaller than the one it is
  // added to, so it takes FastTwoSum (df_add_ord and its variants)
  const float q4 = fmaf(r.hi, 1.0f / 120.0f, 1.0f / 24.0f);
  df q = df_add_f_ord_u(mk(I3H, I3L), __fmul_rn(r.hi, q4));  // 1/6 + r/24 + r^2/120
  q = df_add_to_f_u(0.5f, df_mul(r, q));
  const df p = df_add_ord(r, df_mul(df_sqr(r), q));          // exp(r) - 1
  const ExpEntryDF te = kT2DF[ni & 63];  // one 8-byte load, cached in L1
  const df T = mk(te.hi, te.lo);
  const df e = df_add_ord(T, df_mul(T, p));
  // times 2^m, |m| <= 115
  return df_scale(e, __int_as_float((127 + (ni >> 6)) << 23));
}

__device__ __forceinline__ df df_log(df x) {
  using namespace dfe;
  if (!(x.hi >= 0x1p-100f && x.hi <= 0x1p+100f)) return mk(logf(x.hi), 0.0f);
  const unsigned b = __float_as_uint(x.hi);
  const int j = (int)(((b & 0x7fffffu) + 0x8000u) >> 16);  // nearest multiple of 1/128
  int k = (int)(b >> 23) - 127;
  const df m = df_scale(x, __uint_as_float((unsigned)(127 - k) << 23));  // m.hi in [1, 2)
  const float F = __uint_as_float(0x3f800000u + ((unsigned)j << 16));    // 1 + j/128
  const LogEntryDF E = kLgDF[j];  // one 16-byte load, cached in L1
  const df u = df_mul(two_sum(__fsub_rn(m.hi, F), m.lo), E.rcpF);      // m.hi - F exact
  const float uf = u.hi;
  const float c4 = fmaf(uf, fmaf(uf, fmaf(uf, 1.0f / 7.0f, -1.0f / 6.0f), 0.2f), -0.25f);
  // |u| <= 2^-8: ordered sums as in df_exp
  df c = df_add_f_ord_u(mk(T3H, T3L), __fmul_rn(uf, c4));  // 1/3 - u/4 + u^2/5 - ...
  c = df_add_to_f_u(-0.5f, df_mul(u, c));
  const df l1p = df_add_ord(u, df_mul(df_sqr(u), c));        // log1p(u)
  k += j >= 64 ? 1 : 0;
  const float kf = (float)k;
  // k ln2: k LN1 exact, k LN2 as an exact product, k LN3 rounded
  df kl = two_prod(kf, LN2);
  kl.lo = fmaf(kf, LN3, kl.lo);
  df kln2 = fast_two_sum(__fmul_rn(kf, LN1), kl.hi);
  kln2.lo = __fadd_rn(kln2.lo, kl.lo);
  return df_add(df_add(E.logF, l1p), kln2);
}

}  // namespace osiris_impl
