// Conversions between FP64, FP32 and double-float values by integer
// operations only. On GB300 the FP64 pipe takes one warp instruction per 16
// SM cycles while the integer and FP32 pipes take several per cycle, so the
// FP64 kernels use these to move work that does not need FP64 arithmetic off
// that pipe. Host builds (the CPU tests) take the bit casts from memcpy.
#pragma once

#include <cstdint>
#include <cstring>

#include "df64.cuh"

namespace osiris_impl {

__device__ __forceinline__ long long bits_of(double x) {
#ifdef __CUDA_ARCH__
  return __double_as_longlong(x);
#else
  long long b;
  std::memcpy(&b, &x, sizeof b);
  return b;
#endif
}

__device__ __forceinline__ double double_of(long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double(b);
#else
  double x;
  std::memcpy(&x, &b, sizeof x);
  return x;
#endif
}

// Leading zeros of a non-zero 64-bit value.
__device__ __forceinline__ int clz64(long long v) {
#ifdef __CUDA_ARCH__
  return __clzll(v);
#else
  return __builtin_clzll((unsigned long long)v);
#endif
}

// x as FP32, significand truncated with integer operations only (relative
// error < 2^-23); zero below the FP32 normal range, +-inf above it.
__device__ __forceinline__ float to_float_rz(double x) {
  const long long b = bits_of(x);
  const int hi = (int)(b >> 32);
  const int e = ((hi >> 20) & 0x7ff) - 1023 + 127;
  const int sign = hi & (int)0x80000000;
  if (e <= 0) return __int_as_float(sign);
  if (e >= 255) return __int_as_float(sign | 0x7f800000);
  return __int_as_float(sign | (e << 23) | (int)((b >> 29) & 0x7fffff));
}

// A normal FP32 value as a double, by integer operations only.
__device__ __forceinline__ double float_to_double(float f) {
  const unsigned b = __float_as_uint(f);
  const long long e = (long long)((b >> 23) & 0xff) - 127 + 1023;
  return double_of((long long)(b & 0x80000000u) << 32 | e << 52 |
                   (long long)(b & 0x7fffffu) << 29);
}

// An FP32 value as a double, by integer operations only: zero (and FP32
// denormals, below 1.2e-38) give zero.
__device__ __forceinline__ double float_to_double0(float f) {
  return (__float_as_uint(f) & 0x7f800000u) ? float_to_double(f) : 0.0;
}

// x as a double-float pair by integer operations only: hi is x truncated to
// 24 significant bits, lo the 29 bits below them truncated to 24, so
// hi + lo = x to 2^-46 |x| for |x| in FP32's normal range (hi is zero below
// it and infinite above it); lo is zero where its bits fall below that range.
__device__ __forceinline__ df split_df(double x) {
  const long long b = bits_of(x);
  const float hi = to_float_rz(x);
  const long long m = b & ((1LL << 29) - 1);  // the significand bits below hi's
  const int e = (int)((b >> 52) & 0x7ff);     // biased exponent of x
  const int lead = 63 - clz64(m | 1);         // leading bit of m (m = 0: lo = 0 below)
  const int fe = lead + e - 1075 + 127;       // FP32 biased exponent of that bit
  const unsigned frac = (unsigned)((lead >= 23) ? (m >> (lead - 23)) : (m << (23 - lead)));
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const float lo = (m != 0 && fe > 0) ? __uint_as_float(sign | ((unsigned)fe << 23) |
                                                         (frac & 0x7fffffu))
                                      : 0.0f;
  return mk(hi, lo);
}

}  // namespace osiris_impl
