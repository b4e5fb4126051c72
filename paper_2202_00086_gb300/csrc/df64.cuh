// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of
// two FP32 numbers with |lo| <= ulp(hi)/2, giving a 48-bit significand on the
// FP32 pipe. The building blocks are the error-free transformations of
// Knuth (TwoSum), Dekker (FastTwoSum) and the FMA-based TwoProd; the
// operation sequences follow Dekker (1971) and the double-double arithmetic
// of Hida, Li & Bailey (2001), specialised to pairs of floats.
//
// Every addition and multiplication whose rounding the algorithms rely on is
// written with the __fadd_rn / __fmul_rn intrinsics, which the compiler never
// contracts into an FMA or reassociates; the error terms use explicit fmaf.
#pragma once

#include <cstdint>

namespace osiris_impl {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df mk(float h, float l) {
  df r;
  r.hi = h;
  r.lo = l;
  return r;
}

// a + b exactly as hi + lo (Knuth).
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return mk(s, e);
}

// a + b exactly as hi + lo when |a| >= |b| (Dekker).
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return mk(s, e);
}

// a * b exactly as hi + lo (FMA).
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = fmaf(a, b, -p);
  return mk(p, e);
}

__device__ __forceinline__ df df_from_double(double x) {
  const float h = __double2float_rn(x);
  const float l = __double2float_rn(x - (double)h);
  return mk(h, l);
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df df_neg(df a) { return mk(-a.hi, -a.lo); }

__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// Sum without the final renormalisation: the TwoSum of the leading words is
// exact for any inputs, so hi + lo stays an exact-enough pair (|lo| a few
// ulp(hi)) for further sums and products. Used for intermediate terms whose
// leading word is not itself inspected.
__device__ __forceinline__ df df_add_u(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return s;
}

__device__ __forceinline__ df df_sub_u(df a, df b) { return df_add_u(a, df_neg(b)); }

// df_add_u for operands whose order of magnitude is known, |a.hi| >= |b.hi|:
// Dekker's FastTwoSum of the leading words is then exact too, at half the
// instructions and dependency depth of TwoSum.
__device__ __forceinline__ df df_add_ord_u(df a, df b) {
  df s = fast_two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return s;
}

// df_add for |a.hi| >= |b.hi| (renormalised).
__device__ __forceinline__ df df_add_ord(df a, df b) {
  const df s = df_add_ord_u(a, b);
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_norm(df a) { return fast_two_sum(a.hi, a.lo); }

__device__ __forceinline__ df df_add_f(df a, float b) {
  df s = two_sum(a.hi, b);
  s.lo = __fadd_rn(s.lo, a.lo);
  return fast_two_sum(s.hi, s.lo);
}

// df_add_f without the final renormalisation (see df_add_u).
__device__ __forceinline__ df df_add_f_u(df a, float b) {
  df s = two_sum(a.hi, b);
  s.lo = __fadd_rn(s.lo, a.lo);
  return s;
}

// df_add_f_u for |a.hi| >= |b| (FastTwoSum, see df_add_ord_u).
__device__ __forceinline__ df df_add_f_ord_u(df a, float b) {
  df s = fast_two_sum(a.hi, b);
  s.lo = __fadd_rn(s.lo, a.lo);
  return s;
}

// b + a for a float b with |b| >= |a.hi| (FastTwoSum, see df_add_ord_u).
__device__ __forceinline__ df df_add_to_f_u(float b, df a) {
  df s = fast_two_sum(b, a.hi);
  s.lo = __fadd_rn(s.lo, a.lo);
  return s;
}

// Products are left unrenormalised: TwoProd gives |lo| <= ulp(hi)/2 and the
// cross terms add at most ~2 ulp(hi), so hi + lo is a valid (slightly
// redundant) df; every df_add renormalises. This keeps a product at 4 FP32
// instructions instead of 7 without losing accuracy in the sums it feeds.
__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return p;
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
  df p = two_prod(a.hi, b);
  p.lo = fmaf(a.lo, b, p.lo);
  return p;
}

__device__ __forceinline__ df df_sqr(df a) {
  df p = two_prod(a.hi, a.hi);
  p.lo = fmaf(__fmul_rn(2.0f, a.hi), a.lo, p.lo);
  return p;
}

// a * b + c
__device__ __forceinline__ df df_fma(df a, df b, df c) { return df_add(df_mul(a, b), c); }

// 1 / b: FP32 reciprocal refined by one Newton step, x1 = x0 + x0 (1 - b x0),
// with the residual formed from both words of b. The seed is 1 / b.hi, so the
// result keeps df64 precision only when b.lo is a few ulp(b.hi) at most (the
// error after the step is about (b.lo / b.hi)^2): renormalise a sum that
// cancelled before taking its reciprocal.
__device__ __forceinline__ df df_rcp(df b) {
  const float x0 = __fdividef(1.0f, b.hi);
  float e = fmaf(-b.hi, x0, 1.0f);
  e = fmaf(-b.lo, x0, e);
  return fast_two_sum(x0, __fmul_rn(x0, e));
}

// Multiply by an exact power of two.
__device__ __forceinline__ df df_scale(df a, float p2) {
  return mk(__fmul_rn(a.hi, p2), __fmul_rn(a.lo, p2));
}

// ---------------------------------------------------------------------------
// sin and cos of a df angle. Reduction t = x - k pi/2 with k = rint(2x/pi),
// |t| <= pi/4, using pi/2 split into three floats (the products k * P1 are
// exact for |k| <= 2 and the subtraction from x.hi is exact by Sterbenz).
// Then the Taylor series of sin t and cos t (coefficients (-1)^n / n!): the
// leading terms in df, the terms below 2^-24 of the result in plain FP32.
// ---------------------------------------------------------------------------
namespace dfc {
// pi/2 = P1 + P2 + P3 to about 76 bits (P1 = 0x1.921fb6p+0)
constexpr float P1 = 1.5707963705062866f;
constexpr float P2 = -4.371138828673793e-08f;
constexpr float P3 = -1.7151245100058819e-15f;
// 1/n! as hi + lo (hi = nearest float, lo = nearest float to the remainder)
constexpr float I3H = 0.1666666716337204f, I3L = -4.967053879312289e-09f;
constexpr float I4H = 0.0416666679084301f, I4L = -1.2417634698280722e-09f;
constexpr float I5H = 0.008333333767950535f, I5L = -4.34617203337595e-10f;
constexpr float I6H = 0.0013888889225199819f, I6L = -3.3631094437103215e-11f;
constexpr float I7H = 0.00019841270113829523f, I7L = -2.725596874933456e-12f;
constexpr float I8H = 2.4801587642286904e-05f, I8L = -3.40699609366682e-13f;
constexpr float I9H = 2.7557318844628753e-06f, I9L = 3.793571224297229e-14f;
// 1/n! to FP32 precision for the terms below 2^-24 of the result
constexpr float I10 = 2.755731998149713e-07f, I11 = 2.5052107943679403e-08f,
                I12 = 2.0876755879584152e-09f, I13 = 1.6059044372074283e-10f,
                I14 = 1.147074536050896e-11f, I15 = 7.647163609812713e-13f,
                I16 = 4.7794772561329454e-14f;
}  // namespace dfc

__device__ __forceinline__ void df_sincos(df x, df& s, df& c) {
  using namespace dfc;
  const float k = rintf(x.hi * 0.636619772367581343f);
  // t = x - k (P1 + P2 + P3)
  // x.hi - k P1 and x.lo - k P2 are formed exactly (k P1, k P2 are exact
  // for |k| <= 2 and the first difference is exact by Sterbenz), so t keeps
  // full relative accuracy near the multiples of pi/2 (the poles).
  const float a = fmaf(-k, P1, x.hi);
  const df b = two_sum(x.lo, __fmul_rn(-k, P2));
  df t = two_sum(a, b.hi);
  t.lo = __fadd_rn(t.lo, fmaf(-k, P3, b.lo));
  t = fast_two_sum(t.hi, t.lo);
  // The series steps and the results are left unrenormalised: their only
  // consumers are products and further sums. With u = t^2 <= (pi/4)^2 < 0.62
  // every step adds a term smaller than the one it is added to (the largest
  // ratio is u/2 < 0.31, in cos t = 1 + u (...)), so each takes FastTwoSum.
  const df u = df_sqr(t);
  const float uf = u.hi;
  // sin t = t (1 - u/3! + u^2/5! - ... ): inner terms in FP32
  float ps = fmaf(uf, fmaf(uf, -I15, I13), -I11);  // -1/11! + u/13! - u^2/15!
  df qs = df_add_f_ord_u(mk(I9H, I9L), __fmul_rn(uf, ps));      // 1/9! - u/11! + ...
  qs = df_add_ord_u(mk(-I7H, -I7L), df_mul(u, qs));
  qs = df_add_ord_u(mk(I5H, I5L), df_mul(u, qs));
  qs = df_add_ord_u(mk(-I3H, -I3L), df_mul(u, qs));
  const df st = df_add_ord_u(t, df_mul(df_mul(t, u), qs));
  // cos t = 1 - u/2 + u^2/4! - ...
  float pc = fmaf(uf, fmaf(uf, fmaf(uf, I16, -I14), I12), -I10);  // -1/10! + ...
  df qc = df_add_f_ord_u(mk(I8H, I8L), __fmul_rn(uf, pc));
  qc = df_add_ord_u(mk(-I6H, -I6L), df_mul(u, qc));
  qc = df_add_ord_u(mk(I4H, I4L), df_mul(u, qc));
  qc = df_add_to_f_u(-0.5f, df_mul(u, qc));
  const df ct = df_add_to_f_u(1.0f, df_mul(u, qc));
  // quadrant
  const int q = ((int)k) & 3;
  if (q == 0) {
    s = st;
    c = ct;
  } else if (q == 1) {
    s = ct;
    c = df_neg(st);
  } else if (q == 2) {
    s = df_neg(st);
    c = df_neg(ct);
  } else {
    s = df_neg(ct);
    c = st;
  }
}

}  // namespace osiris_impl
