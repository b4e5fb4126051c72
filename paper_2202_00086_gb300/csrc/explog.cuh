// Table-driven exp and log in double precision, for the q-metric's powers
// f^q and X^k (Appendix A), which cost most of its evaluation when taken
// from the library.
//
// exp, after P. T. P. Tang, "Table-driven implementation of the exponential
// function in IEEE floating-point arithmetic", ACM TOMS 15 (1989):
//   y = (64 m + j) ln2/64 + r with |r| <= ln2/128, and
//   exp(y) = 2^m 2^(j/64) (1 + p(r)), p(r) = exp(r) - 1 by its Taylor series
//   through r^5 (truncation below 2e-17 relative).
// log, after P. T. P. Tang, "Table-driven implementation of the logarithm
// function in IEEE floating-point arithmetic", ACM TOMS 16 (1990):
//   x = 2^k m with m in [1, 2), F = 1 + j/128 the breakpoint nearest m,
//   log x = k ln2 + log F + log1p(u), u = (m - F)/F, |u| <= 2^-8, and
//   log1p(u) by its Taylor series through u^7 (truncation below 1e-20).
//   Breakpoints F >= 1.5 are stored as log(F/2) with k + 1, so that for x
//   just below 1 the first two terms vanish exactly and the result keeps its
//   relative accuracy.
// The tables hold the doubles nearest 2^(j/64), log F (or log(F/2)) and 1/F
// (explog_tables.h, written by gen_explog_tables.py at 200-bit precision);
// device code copies them into shared memory once per block. Arguments
// outside the reduced forms' range
// (exp: |y| >= 700 or NaN; log: x outside [2^-1000, 2^1000] or NaN) go to the
// library functions. The higher-order parts of the two series,
// exp(r) - 1 - r (< 1.5e-5) and log1p(u) - u (< 7.7e-6), are small against
// the results, so they are formed in double-float on the FP32 pipe
// (convert.cuh, df64.cuh; their own leading terms in two words) and added to
// r or u in FP64: 7 FP64 instructions for exp and 8 for log instead of 10 and
// 13. Both stay within 2 ulp of the
// exact value (measured worst cases are in tests/test_explog_host.py, where
// log(F/2) and log1p(u) partly cancel). The functions also compile as host
// C++, which is how that bound is tested, against mpmath and libm.
#pragma once

#include <cmath>
#include <cstring>

#include "explog_tables.h"

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

#include "convert.cuh"

namespace osiris_explog {

constexpr int kExpN = 64;      // 2^(j/64), j = 0..63
constexpr int kLogN = 129;     // F_j = 1 + j/128, j = 0..128
constexpr int kLogHalf = 64;   // from j = 64 (F >= 1.5): log(F/2), exponent k + 1

struct LogEntry {
  double logF;  // log F_j, or log(F_j / 2) for j >= kLogHalf
  double rcpF;  // 1 / F_j
};

struct Tables {  // the block's shared-memory copy
  double t2[kExpN];
  LogEntry lg[kLogN];
};

__host__ __device__ __forceinline__ long long to_bits(double x) {
#ifdef __CUDA_ARCH__
  return __double_as_longlong(x);
#else
  long long b;
  std::memcpy(&b, &x, sizeof b);
  return b;
#endif
}

__host__ __device__ __forceinline__ double from_bits(long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double(b);
#else
  double x;
  std::memcpy(&x, &b, sizeof x);
  return x;
#endif
}

#ifdef __CUDACC__
#define OSIRIS_EXPLOG_STORAGE static __constant__
#else
#define OSIRIS_EXPLOG_STORAGE static const
#endif
OSIRIS_EXPLOG_STORAGE double kT2[kExpN] = {OSIRIS_EXPLOG_T2};
OSIRIS_EXPLOG_STORAGE LogEntry kLg[kLogN] = {OSIRIS_EXPLOG_LG};
#undef OSIRIS_EXPLOG_STORAGE

// ln2/64 and 64/ln2 as doubles, and ln2/64 - (its double) for the second
// step of the reduction; ln2 and its remainder likewise.
constexpr double kInvL = 0x1.71547652b82fep+6;
constexpr double kL1 = 0x1.62e42fefa39efp-7;
constexpr double kL2 = 0x1.abc9e3b39803fp-62;
constexpr double kLn2Hi = 0x1.62e42fefa39efp-1;
constexpr double kLn2Lo = 0x1.abc9e3b39803fp-56;
// adding 1.5 * 2^52 rounds to an integer held in the low significand bits
constexpr double kShift = 0x1.8p52;
constexpr long long kShiftBits = 0x4338000000000000LL;

// 1/3 as a float pair, for the log1p series
constexpr float kThirdH = 0.3333333432674408f, kThirdL = -9.934107758624577e-09f;

__device__ __forceinline__ double exp_tab(double y, const double* t2) {
  using namespace osiris_impl;
  if (!(fabs(y) < 700.0)) return exp(y);
  const double t = fma(y, kInvL, kShift);
  const int n = (int)(to_bits(t) & 0xffffffffLL);  // y * 64/ln2 rounded, mod 2^32
  const double nd = t - kShift;
  const double r = fma(-nd, kL2, fma(-nd, kL1, y));
  // exp(r) - 1 = r + c, c = r^2 (1/2 + r/6 + r^2/24 + r^3/120), in double-float:
  // the r/6 term as a product with 1/6 in two words, the rest in FP32
  const df rd = split_df(r);
  const float rf = rd.hi;
  const float small = __fmul_rn(__fmul_rn(rf, rf), fmaf(rf, 1.0f / 120.0f, 1.0f / 24.0f));
  const df q = df_add_f_u(df_add_f_u(df_mul(rd, mk(dfc::I3H, dfc::I3L)), small), 0.5f);
  const df c = df_mul(df_sqr(rd), q);
  const double p = (r + float_to_double0(c.hi)) + float_to_double0(c.lo);
  const double T = t2[n & (kExpN - 1)];
  const double e = fma(T, p, T);  // in [0.99, 2.02): scaling by 2^m stays normal
  return from_bits(to_bits(e) + (long long)(n >> 6) * (1LL << 52));
}

__device__ __forceinline__ double log_tab(double x, const LogEntry* lg) {
  using namespace osiris_impl;
  if (!(x >= 0x1p-1000 && x <= 0x1p+1000)) return log(x);
  const long long b = to_bits(x);
  const int hi = (int)(b >> 32);
  const double m = from_bits((b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
  const int j = ((hi & 0xfffff) + 0x1000) >> 13;  // nearest multiple of 1/128, 0..128
  const double F = from_bits(0x3ff0000000000000LL + ((long long)j << 45));
  const LogEntry E = lg[j];
  const double u = (m - F) * E.rcpF;  // m - F is exact
  // log1p(u) = u + c, c = u^2 (-1/2 + u/3 - u^2/4 + u^3/5 - u^4/6 + u^5/7), in
  // double-float. The result is ~u, so c needs ~2^-53 / |u| relative accuracy:
  // the u/3 and u^2/4 terms in two words, from u^3 on in FP32.
  const df ud = split_df(u);
  const float uf = ud.hi;
  const df usq = df_sqr(ud);
  const float small = __fmul_rn(__fmul_rn(uf, __fmul_rn(uf, uf)),
                                fmaf(uf, fmaf(uf, 1.0f / 7.0f, -1.0f / 6.0f), 1.0f / 5.0f));
  const df q = df_add_f_u(
      df_add_f_u(df_add_u(df_mul(ud, mk(kThirdH, kThirdL)), df_scale(usq, -0.25f)), small),
      -0.5f);
  const df c = df_mul(usq, q);
  const double l1p = (u + float_to_double0(c.hi)) + float_to_double0(c.lo);
  const int k = (hi >> 20) - 1023 + (j >= kLogHalf ? 1 : 0);
  const double kd = from_bits(kShiftBits + k) - kShift;
  return fma(kd, kLn2Hi, E.logF) + fma(kd, kLn2Lo, l1p);
}

}  // namespace osiris_explog
