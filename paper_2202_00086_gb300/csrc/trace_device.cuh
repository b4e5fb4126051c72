// Device side of the backward ray tracer: Hamilton's equations for null
// geodesics in Kerr space-time (Sec. 2.1, Sec. 4.3), adaptive Cash-Karp 4(5)
// steps (Sec. 3.1), the |H| constraint error, stopping surfaces (Sec. 4.1,
// Sec. 5) and the per-ray observables.
//
// Execution model (one ray per lane):
//   Every lane of a warp runs the same loop body each iteration: ONE
//   Cash-Karp attempt from its current state with its own step length.
//   What the lane does with the result depends on its mode:
//     INTEGRATE  accept/reject under the error controller; an accepted step
//                that crosses a stopping surface switches the lane to LOCATE
//     LOCATE     the attempt is a trial step length inside the bracket of the
//                crossing (Illinois-modified regula falsi); on convergence the
//                ray finishes (or, for an equatorial crossing outside the
//                disk, resumes integrating)
//     IDLE       no ray (finished; persistent grids refill it from the queue)
//   So surface location and refills never serialise a warp behind one lane:
//   the expensive part (six evaluations of the equations of motion) is the
//   same instruction stream for every lane.
#pragma once

#include <cstdint>

#include "convert.cuh"
#include "df64.cuh"
#include "explog.cuh"
#include "osiris_internal.h"

namespace osiris_impl {

// ---------------------------------------------------------------------------
// Cash-Karp 4(5) tableau (Cash & Karp 1990, the RKCK45 scheme of Sec. 3.1).
// ---------------------------------------------------------------------------
namespace ck {
constexpr double A21 = 1.0 / 5.0;
constexpr double A31 = 3.0 / 40.0, A32 = 9.0 / 40.0;
constexpr double A41 = 3.0 / 10.0, A42 = -9.0 / 10.0, A43 = 6.0 / 5.0;
constexpr double A51 = -11.0 / 54.0, A52 = 5.0 / 2.0, A53 = -70.0 / 27.0, A54 = 35.0 / 27.0;
constexpr double A61 = 1631.0 / 55296.0, A62 = 175.0 / 512.0, A63 = 575.0 / 13824.0,
                 A64 = 44275.0 / 110592.0, A65 = 253.0 / 4096.0;
// fifth-order weights (propagated solution); stages 2 and 5 have weight 0
constexpr double B1 = 37.0 / 378.0, B3 = 250.0 / 621.0, B4 = 125.0 / 594.0,
                 B6 = 512.0 / 1771.0;
// fifth minus embedded fourth order (error estimate weights), exact rationals
constexpr double D1 = -277.0 / 64512.0, D3 = 6925.0 / 370944.0, D4 = -6925.0 / 202752.0,
                 D5 = -277.0 / 14336.0, D6 = 277.0 / 7084.0;
}  // namespace ck

// Dormand-Prince 5(4) tableau (Dormand & Prince 1980, the RKDP45 scheme of
// Sec. 3.1). Seven stages; the seventh is evaluated at the fifth-order
// solution, so it is the first stage of the next step (first same as last).
namespace dp {
constexpr double A21 = 1.0 / 5.0;
constexpr double A31 = 3.0 / 40.0, A32 = 9.0 / 40.0;
constexpr double A41 = 44.0 / 45.0, A42 = -56.0 / 15.0, A43 = 32.0 / 9.0;
constexpr double A51 = 19372.0 / 6561.0, A52 = -25360.0 / 2187.0, A53 = 64448.0 / 6561.0,
                 A54 = -212.0 / 729.0;
constexpr double A61 = 9017.0 / 3168.0, A62 = -355.0 / 33.0, A63 = 46732.0 / 5247.0,
                 A64 = 49.0 / 176.0, A65 = -5103.0 / 18656.0;
// fifth-order weights = the seventh row; b2 = b7 = 0
constexpr double B1 = 35.0 / 384.0, B3 = 500.0 / 1113.0, B4 = 125.0 / 192.0,
                 B5 = -2187.0 / 6784.0, B6 = 11.0 / 84.0;
// fifth minus embedded fourth order, exact rationals
constexpr double D1 = 71.0 / 57600.0, D3 = -71.0 / 16695.0, D4 = 71.0 / 1920.0,
                 D5 = -17253.0 / 339200.0, D6 = 22.0 / 525.0, D7 = -1.0 / 40.0;
}  // namespace dp

// pi/2 split in two doubles: (PIO2_HI - theta) + PIO2_LO has the sign of
// cos(theta) for theta in (-pi/2, 3pi/2), and equals it to first order near
// the equator.
constexpr double PIO2_HI = 1.5707963267948966;
constexpr double PIO2_LO = 6.123233995736766e-17;
constexpr double TWO_PI = 6.283185307179586;
constexpr double PI_D = 3.141592653589793;

enum : int { MODE_IDLE = 0, MODE_INTEGRATE = 1, MODE_LOCATE = 2, MODE_DONE = 3 };
enum : int { SURF_EQUATOR = 0, SURF_CAPTURE = 1, SURF_ESCAPE = 2 };

struct State {  // evolved coordinates and momenta (t does not feed back; not integrated)
  double r, th, ph, pr, pth;
};

// Per-ray constants of the Hamiltonian (Kerr: a and its products; q-metric:
// q and kap = q (2 + q)).
struct RayK {
  double a, a2, aE, aL, E, L;
  double E2;  // 2E
  double q, kap;
};

// ---------------------------------------------------------------------------
// FP64 sine/cosine and reciprocal with few FP64-pipe instructions.
//
// GB300's FP64 pipe takes one warp instruction per 16 SM cycles (a fused
// multiply-add; a separate multiply or add takes 19), while its FP32, integer
// and shared-memory pipes are nearly idle in this kernel; the helpers below
// move the argument reduction, table look-up, seeds and the small sine/cosine
// corrections onto those pipes and keep only the accuracy-critical FP64
// arithmetic.
//
// sincos_tab: theta = N_k + x, where the node N_k is the double nearest to
// k pi/512 (the node index found in FP32), so that x = theta - N_k is exact
// (Sterbenz) and |x| <= pi/1024 (+ FP32 rounding). sin and cos of the node
// itself (not of k pi/512) come from a per-block shared-memory table filled
// with the library sincos; sin x - x and cos x - 1 from their Taylor series
// (truncation below 0.01 ulp at |x| = 0.0031):
//   sin x - x = x^3 (-1/6 + x^2/120),   cos x - 1 = x^2 (-1/2 + x^2/24),
//   sin theta = (S_k + C_k x) + [C_k (sin x - x) + S_k (cos x - 1)],
//   cos theta = (C_k - S_k x) + [C_k (cos x - 1) - S_k (sin x - x)].
// The bracketed corrections are at most 5e-6 of the result and need only
// ~1e-11 relative accuracy, so they are formed in double-float on the FP32
// pipe from x split into two floats by integer operations; the FP64 pipe does
// x itself, C_k x added to S_k and the correction's two words added on: 7 FP64
// instructions for both results, each within ~1.5 ulp. The table covers theta
// in [-pi/16, 17 pi/16], which holds every ray except one passing almost
// exactly over a pole; outside it the library sincos is used.
// ---------------------------------------------------------------------------
constexpr int kTrigPerPi = 512;                      // nodes per pi
constexpr int kTrigFirst = -kTrigPerPi / 16;         // node index of the first entry
constexpr int kTrigNodes = kTrigPerPi + 2 * (kTrigPerPi / 16) + 1;

struct TrigTable {
  double2 sc[kTrigNodes];  // sin N_k, cos N_k
  float4 scf[kTrigNodes];  // the same as double-float pairs (sin hi, lo, cos hi, lo)
  double n[kTrigNodes];    // N_k
};

__device__ __forceinline__ TrigTable& trig_table() {
  __shared__ TrigTable table;
  return table;
}

// Fill the block's table (all threads of the block, before any divergence).
__device__ __forceinline__ void trig_table_init() {
  constexpr double STEP = 3.141592653589793116 / kTrigPerPi;  // exact: pi rounded / 2^9
  TrigTable& t = trig_table();
  for (int i = threadIdx.x; i < kTrigNodes; i += blockDim.x) {
    const double n = (double)(i + kTrigFirst) * STEP;
    double s, c;
    sincos(n, &s, &c);
    t.sc[i] = make_double2(s, c);
    const float sh = (float)s, ch = (float)c;
    t.scf[i] = make_float4(sh, (float)(s - (double)sh), ch, (float)(c - (double)ch));
    t.n[i] = n;
  }
  __syncthreads();
}

// The block's copy of the exp/log breakpoint tables (explog.cuh), filled by
// all threads of the block before any divergence.
__device__ __forceinline__ osiris_explog::Tables& explog_table() {
  __shared__ osiris_explog::Tables table;
  return table;
}

__device__ __forceinline__ void explog_table_init() {
  osiris_explog::Tables& t = explog_table();
  for (int i = threadIdx.x; i < osiris_explog::kLogN; i += blockDim.x) {
    if (i < osiris_explog::kExpN) t.t2[i] = osiris_explog::kT2[i];
    t.lg[i] = osiris_explog::kLg[i];
  }
  __syncthreads();
}



// a b and a + c issued as fused multiply-adds: fma(a, b, -0) = a b and
// fma(a, 1, c) = a + c exactly (one rounding each, the same result bit for
// bit, signed zeros included). The -0 and 1 come from constant memory, whose
// values no compiler pass may assume, so the instruction stays a fused
// multiply-add instead of being folded back into a multiply or an add.
#ifdef __CUDACC__
static __constant__ double kFmaNegZero = -0.0;
static __constant__ double kFmaOne = 1.0;
#endif

__device__ __forceinline__ double mul_as_fma(double a, double b) {
#ifdef __CUDA_ARCH__
  double r;
  asm("fma.rn.f64 %0, %1, %2, %3;" : "=d"(r) : "d"(a), "d"(b), "d"(kFmaNegZero));
  return r;
#else
  return a * b;
#endif
}

__device__ __forceinline__ double add_as_fma(double a, double c) {
#ifdef __CUDA_ARCH__
  double r;
  asm("fma.rn.f64 %0, %1, %2, %3;" : "=d"(r) : "d"(a), "d"(kFmaOne), "d"(c));
  return r;
#else
  return a + c;
#endif
}

__device__ __forceinline__ float mul_as_fma(float a, float b) { return a * b; }
__device__ __forceinline__ float add_as_fma(float a, float c) { return a + c; }




__device__ __forceinline__ void sincos_tab(double th, double& s, double& c) {
  using namespace dfc;
  // nearest node in FP32: 1.5 * 2^23 added to round to an integer
  const float tk = fmaf(to_float_rz(th), (float)(kTrigPerPi / 3.14159265358979323846),
                        12582912.0f);
  const int idx = (__float_as_int(tk) - 0x4B400000) - kTrigFirst;
  if ((unsigned)idx >= (unsigned)kTrigNodes) {  // also NaN / inf
    sincos(th, &s, &c);
    return;
  }
  const TrigTable& t = trig_table();
  const double2 sc = t.sc[idx];
  const float4 scf = t.scf[idx];
  const double x = th - t.n[idx];  // exact
  // the corrections in double-float
  const df xd = split_df(x);
  const df u = df_sqr(xd);                                                    // x^2
  const df q = df_add_f_u(mk(-I3H, -I3L), __fmul_rn(u.hi, 1.0f / 120.0f));    // -1/6 + x^2/120
  const df ds = df_mul(df_mul(xd, u), q);                                     // sin x - x
  const df cm = df_add_f_u(df_scale(u, -0.5f),
                           __fmul_rn(__fmul_rn(u.hi, u.hi), 1.0f / 24.0f));   // cos x - 1
  const df S = mk(scf.x, scf.y), C = mk(scf.z, scf.w);
  const df corr_s = df_add_u(df_mul(C, ds), df_mul(S, cm));
  const df corr_c = df_sub_u(df_mul(C, cm), df_mul(S, ds));
  s = fma(sc.y, x, sc.x + float_to_double0(corr_s.hi)) + float_to_double0(corr_s.lo);
  c = fma(-sc.x, x, sc.y + float_to_double0(corr_c.hi)) + float_to_double0(corr_c.lo);
}

// max |H - H0| kept as the bit pattern of a non-negative double: |v| and the
// maximum are integer operations; NaN is ignored like fmax does.
__device__ __forceinline__ void track_abs_H(long long& max_bits, double twoH, double H0) {
  const long long b = __double_as_longlong(fma(0.5, twoH, -H0)) & 0x7fffffffffffffffLL;
  if (b <= 0x7ff0000000000000LL && b > max_bits) max_bits = b;
}

// 1/d: FP32 seed x0 (|x0 d - 1| < 2^-21), then one Newton step with the
// cubic term, x0 (1 + e + e^2) with e = 1 - d x0, relative error e^3 plus
// the final rounding (3 FP64 instructions). Outside the FP32 range: 1/d.
__device__ __forceinline__ double rcp64(double d) {
  const long long b = __double_as_longlong(d);
  const int e = (int)((b >> 52) & 0x7ff) - 1023 + 127;
  if (e < 2 || e > 252) return 1.0 / d;
  const float f = __int_as_float((int)((b >> 32) & 0x80000000) | (e << 23) |
                                 (int)((b >> 29) & 0x7fffff));
  float rf;
#ifdef __CUDA_ARCH__
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(f));
#else
  rf = 1.0f / f;  // host builds of this header (CPU tests): a correctly rounded seed
#endif
  const double x0 = float_to_double(rf);
  const double eps = fma(-d, x0, 1.0);
  return fma(x0, fma(eps, eps, eps), x0);
}

// ---------------------------------------------------------------------------
// Hamilton's equations in separated form.
//
// With p_t = -E, p_phi = L, the Kerr Hamiltonian H = 1/2 g^{mu nu} p_mu p_nu
// (Eq. ligH) on the inverse of the metric of Eq. Kerr can be written
//   H = N / (2 Sigma),
//   N = Delta p_r^2 + p_theta^2 + W^2 - P^2 / Delta,
//   P = (r^2 + a^2) E - a L,   W = L / sin(theta) - a E sin(theta).
// Its exact derivatives (no use of H = 0, so the flow is the paper's flow
// everywhere, also off the constraint surface) give, with u = P / Delta,
//   r'       =  Delta p_r / Sigma
//   theta'   =  p_theta / Sigma
//   phi'     =  (W / sin + a u) / Sigma
//   p_r'     =  [ r N / Sigma - (r - 1)(p_r^2 + u^2) + 2 r E u ] / Sigma
//   p_theta' =  cos [ W (L / sin^2 + a E) - a^2 sin N / Sigma ] / Sigma
// which are the component equations of Sec. 2.1 after the common factors
// are collected. One reciprocal of Delta Sigma sin(theta) yields all three
// reciprocals. The outputs are the bracketed terms (the derivatives times
// Sigma) and scale = 1 / Sigma, which the stepper folds into its tableau
// coefficients; products are shared where the algebra allows (Sigma from
// r^2 + a^2 - a^2 sin^2, p_r' as Y + r (X - Y) with X = 2H + 2 E u and
// Y = p_r^2 + u^2, L / sin reused). twoH receives 2H = N / Sigma at the
// evaluation point.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void rhs64(const RayK& K, double r, double th, double pr, double pth,
                                      double& dr, double& dth, double& dph, double& dpr,
                                      double& dpth, double& twoH, double& scale) {
  double s, c;
  sincos_tab(th, s, c);
  const double ra2 = fma(r, r, K.a2);  // r^2 + a^2
  const double a2s = K.a2 * s;
  const double Delta = fma(r, r - 2.0, K.a2);
  // Sigma = r^2 + a^2 cos^2 = (r^2 + a^2) - a^2 sin^2 (no cancellation: r > a)
  const double Sigma = fma(-a2s, s, ra2);
  const double P = fma(ra2, K.E, -K.aL);
  const double DS = Delta * Sigma;
  const double inv = rcp64(DS * s);
  const double sinv = s * inv;  // 1 / (Delta Sigma)
  const double iSig = Delta * sinv;
  const double iDel = Sigma * sinv;
  const double is = DS * inv;
  const double Lis = K.L * is;  // L / sin
  const double W = fma(-K.aE, s, Lis);
  const double u = P * iDel;
  const double Dpr = Delta * pr;
  const double N = fma(Dpr, pr, fma(pth, pth, fma(W, W, -P * u)));
  const double NiS = N * iSig;
  // Every derivative carries the factor 1/Sigma; it is returned separately
  // (scale) and folded into the stepper's tableau coefficients.
  dr = Dpr;
  dth = pth;
  dph = fma(W, is, K.a * u);
  // -dH/dr: (1 - r) Y + r X = Y + r (X - Y), Y = u^2 + p_r^2, X = 2H + 2E u
  const double Y = fma(u, u, pr * pr);
  dpr = fma(r, fma(K.E2, u, NiS) - Y, Y);
  // -dH/dtheta: cos (W (L / sin^2 + a E) - a^2 sin 2H)
  dpth = c * fma(W, fma(Lis, is, K.aE), -a2s * NiS);
  scale = iSig;
  twoH = NiS;
}

// ---------------------------------------------------------------------------
// Hamilton's equations on the q-metric (Appendix A, Eq. q-metric, signature
// -+++, m = 1). The metric is diagonal, so with f = 1 - 2/r, D = r^2 - 2r,
// X = 1 + sin^2 / D, k = q (2 + q):
//   g^tt = -f^-(1+q), g^rr = f^(1+q) X^k, g^thth = f^q X^k / r^2,
//   g^phph = f^q / (r^2 sin^2),
// and each derivative is g^{mu mu} times its logarithmic derivative
// (d ln f / dr = 2/D, d ln X / dr = -sin^2 (2r - 2) / (D^2 X),
//  d ln X / dtheta = 2 sin cos / (D X)).
// The powers f^q and X^k come from the table-driven exp and log of
// explog.cuh (about a third of the library's FP64 instructions).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void rhs_q64(const RayK& K, double r, double th, double pr,
                                        double pth, double& dr, double& dth, double& dph,
                                        double& dpr, double& dpth, double& twoH, double& scale) {
  scale = 1.0;
  double s, c;
  sincos_tab(th, s, c);
  // four reciprocals (1/D, 1/X, 1/sin^2, 1/(f f^q)) serve every quotient:
  // 1/r = (r - 2)/D, and f = (r - 2)/r keeps its relative accuracy at r -> 2
  const double rm2 = r - 2.0;
  const double iD = rcp64(r * rm2);
  const double ir = rm2 * iD;
  const double f = rm2 * ir;
  const double s2 = s * s;
  const double is2 = rcp64(s2);
  const double X = fma(s2, iD, 1.0);
  const double iX = rcp64(X);
  const osiris_explog::Tables& T = explog_table();
  const double fq = osiris_explog::exp_tab(K.q * osiris_explog::log_tab(f, T.lg), T.t2);
  const double Xk = osiris_explog::exp_tab(K.kap * osiris_explog::log_tab(X, T.lg), T.t2);
  const double ir2 = ir * ir;
  const double ffq = f * fq;
  const double fXk = fq * Xk;
  const double gtt = -rcp64(ffq);
  const double grr = f * fXk;
  const double gthth = fXk * ir2;
  const double gpp = fq * ir2 * is2;
  dr = grr * pr;
  dth = gthth * pth;
  dph = gpp * K.L;
  // the four terms of 2H
  const double Ht = gtt * (K.E * K.E), Hr = dr * pr, Hth = dth * pth, Hph = dph * K.L;
  twoH = (Ht + Hr) + (Hth + Hph);
  // -dH/dr = -1/2 sum_mu (d ln g^mumu / dr) H_mu, collected by logarithmic
  // derivative: -1/2 [(1+q) d ln f (Hr - Ht) + k d ln X (Hr + Hth)
  //                   + (q d ln f - 2/r) (Hth + Hph)]
  const double iDX = iD * iX;
  const double a1 = fma(-K.q, iD, -iD);                 // -(1+q)/D
  const double a2 = K.kap * s2 * (r - 1.0) * iD * iDX;  // k sin^2 (r-1) / (D^2 X)
  const double a3 = fma(-K.q, iD, ir);                  // 1/r - q/D
  dpr = fma(a1, Hr - Ht, fma(a2, Hr + Hth, a3 * (Hth + Hph)));
  // -dH/dtheta = -1/2 (k d ln X/dtheta (Hr + Hth) - 2 (cos/sin) Hph)
  //            = sin cos (Hph / sin^2 - k (Hr + Hth) / (D X))
  dpth = (c * s) * fma(-K.kap * iDX, Hr + Hth, Hph * is2);
}

// Metric policies for the FP64 steppers.
#ifndef OSIRIS_FP64_MAXREGS
#define OSIRIS_FP64_MAXREGS 255
#endif

struct KerrMetric {
  static constexpr bool kTrigTable = true;  // rhs64 reads the block's sincos table
  static constexpr bool kExpLogTable = false;
  // No register cap (the compiler takes ~200, two blocks of 128 threads per
  // SM): measured on the 12 x 1024^2 Kerr set, 3.09 Mrays/s uncapped against
  // 2.95 at 168 registers (three blocks) and 2.90 at 152 or 128 (three or
  // four blocks). The FP64 pipe needs the scheduling freedom more than warps.
  static constexpr int kMaxRegs = OSIRIS_FP64_MAXREGS;
  static __device__ __forceinline__ void rhs(const RayK& K, double r, double th, double pr,
                                             double pth, double& dr, double& dth, double& dph,
                                             double& dpr, double& dpth, double& twoH,
                                             double& scale) {
    rhs64(K, r, th, pr, pth, dr, dth, dph, dpr, dpth, twoH, scale);
  }
};
struct QMetric {
  static constexpr bool kTrigTable = true;  // rhs_q64 reads the block's sincos table
  static constexpr bool kExpLogTable = true;  // and the exp/log tables
  static constexpr int kMaxRegs = OSIRIS_FP64_MAXREGS;
  static __device__ __forceinline__ void rhs(const RayK& K, double r, double th, double pr,
                                             double pth, double& dr, double& dth, double& dph,
                                             double& dpr, double& dpth, double& twoH,
                                             double& scale) {
    rhs_q64(K, r, th, pr, pth, dr, dth, dph, dpr, dpth, twoH, scale);
  }
};

// One evaluation of Hamilton's equations in scaled form: the derivative of
// the evolved components (r, theta, phi, p_r, p_theta) is scale * (r, th, ph,
// pr, pth); twoH = 2H at the evaluation point.
struct Deriv {
  double r, th, ph, pr, pth;
  double scale, twoH;
};

template <class Met = KerrMetric>
__device__ __forceinline__ void rhs64_at(const RayK& K, double r, double th, double pr,
                                         double pth, Deriv& k) {
  Met::rhs(K, r, th, pr, pth, k.r, k.th, k.ph, k.pr, k.pth, k.twoH, k.scale);
}

template <class Met = KerrMetric>
__device__ __forceinline__ void rhs64_at(const RayK& K, const State& y, Deriv& k) {
  rhs64_at<Met>(K, y.r, y.th, y.pr, y.pth, k);
}

// 2H at a state (used once per ray for the terminal point).
template <class Met = KerrMetric>
__device__ __forceinline__ double twoH64(const RayK& K, const State& y) {
  Deriv k;
  rhs64_at<Met>(K, y, k);
  return k.twoH;
}

// Embedded Runge-Kutta attempt of length h from y with the tableau T (FP64
// everywhere): o = fifth-order result, d = fifth minus fourth order. The
// stage derivative k_j = scale_j * k~_j enters every sum through the
// coefficient T.a[s][j] * (h scale_j), so the evaluations never multiply their
// outputs by 1/Sigma; the stage inputs and o are accumulated directly onto y
// (a few ulp of |y| per step, far below the truncation error at any usable
// tolerance). phi is cyclic: its stage values are never needed, only its
// increment. With FSAL the last stage is evaluated at o itself and k[NS - 1]
// is the first stage of the next step.
template <int NS>
struct Tableau64 {
  double a[NS][NS];  // a[s][j], j < s
  double b[NS];      // fifth-order weights
  double e[NS];      // fifth minus embedded fourth order
};

// Stages 1 .. NS-1 (stage 0, k[0], is given), o and d. FSAL: the last
// stage is evaluated at o.
template <class Met, int NS, bool FSAL>
__device__ __forceinline__ void rk_attempt64(const Tableau64<NS>& T, const RayK& K,
                                             const State& y, double h, Deriv (&k)[NS],
                                             State& o, State& d) {
  double w[NS];
  w[0] = h * k[0].scale;
  constexpr int NI = FSAL ? NS - 1 : NS;  // stages whose input is a stage sum
#pragma unroll
  for (int s = 1; s < NI; ++s) {
    double ir = y.r, it = y.th, ip = y.pr, iq = y.pth;
#pragma unroll
    for (int j = 0; j < s; ++j) {
      if (T.a[s][j] != 0.0) {
        const double c = T.a[s][j] * w[j];
        ir = fma(c, k[j].r, ir);
        it = fma(c, k[j].th, it);
        ip = fma(c, k[j].pr, ip);
        iq = fma(c, k[j].pth, iq);
      }
    }
    rhs64_at<Met>(K, ir, it, ip, iq, k[s]);
    w[s] = h * k[s].scale;
  }
  o = y;
#pragma unroll
  for (int j = 0; j < NI; ++j) {
    if (T.b[j] != 0.0) {
      const double c = T.b[j] * w[j];
      o.r = fma(c, k[j].r, o.r);
      o.th = fma(c, k[j].th, o.th);
      o.ph = fma(c, k[j].ph, o.ph);
      o.pr = fma(c, k[j].pr, o.pr);
      o.pth = fma(c, k[j].pth, o.pth);
    }
  }
  if (FSAL) {
    rhs64_at<Met>(K, o, k[NS - 1]);
    w[NS - 1] = h * k[NS - 1].scale;
  }
  const double c0 = T.e[0] * w[0];
  d.r = c0 * k[0].r;
  d.th = c0 * k[0].th;
  d.ph = c0 * k[0].ph;
  d.pr = c0 * k[0].pr;
  d.pth = c0 * k[0].pth;
#pragma unroll
  for (int j = 1; j < NS; ++j) {
    if (T.e[j] != 0.0) {
      const double c = T.e[j] * w[j];
      d.r = fma(c, k[j].r, d.r);
      d.th = fma(c, k[j].th, d.th);
      d.ph = fma(c, k[j].ph, d.ph);
      d.pr = fma(c, k[j].pr, d.pr);
      d.pth = fma(c, k[j].pth, d.pth);
    }
  }
}

// One Cash-Karp attempt of length h from y (Sec. 3.1, RKCK45).
template <class Met = KerrMetric>
__device__ __forceinline__ void ck_step64(const RayK& K, const State& y, double h, State& o,
                                          State& d, double& twoH) {
  constexpr Tableau64<6> T = {
      {{0, 0, 0, 0, 0, 0},
       {ck::A21, 0, 0, 0, 0, 0},
       {ck::A31, ck::A32, 0, 0, 0, 0},
       {ck::A41, ck::A42, ck::A43, 0, 0, 0},
       {ck::A51, ck::A52, ck::A53, ck::A54, 0, 0},
       {ck::A61, ck::A62, ck::A63, ck::A64, ck::A65, 0}},
      {ck::B1, 0, ck::B3, ck::B4, 0, ck::B6},
      {ck::D1, 0, ck::D3, ck::D4, ck::D5, ck::D6}};
  Deriv k[6];
  rhs64_at<Met>(K, y, k[0]);
  twoH = k[0].twoH;
  rk_attempt64<Met, 6, false>(T, K, y, h, k, o, d);
}

// One Dormand-Prince attempt of length h from y given k1 = f(y) (Sec. 3.1,
// RKDP45): six new evaluations; k7 = f(o) is the first stage of the next
// step if this one is accepted.
template <class Met = KerrMetric>
__device__ __forceinline__ void dp_step64(const RayK& K, const State& y, double h,
                                          const Deriv& k1, State& o, State& d, Deriv& k7) {
  constexpr Tableau64<7> T = {
      {{0, 0, 0, 0, 0, 0, 0},
       {dp::A21, 0, 0, 0, 0, 0, 0},
       {dp::A31, dp::A32, 0, 0, 0, 0, 0},
       {dp::A41, dp::A42, dp::A43, 0, 0, 0, 0},
       {dp::A51, dp::A52, dp::A53, dp::A54, 0, 0, 0},
       {dp::A61, dp::A62, dp::A63, dp::A64, dp::A65, 0, 0},
       {0, 0, 0, 0, 0, 0, 0}},  // the seventh stage is evaluated at o
      {dp::B1, 0, dp::B3, dp::B4, dp::B5, dp::B6, 0},
      {dp::D1, 0, dp::D3, dp::D4, dp::D5, dp::D6, dp::D7}};
  Deriv k[7];
  k[0] = k1;
  rk_attempt64<Met, 7, true>(T, K, y, h, k, o, d);
  k7 = k[6];
}

// True when x is +-inf or NaN (exponent bits all set); integer test only.
__device__ __forceinline__ bool not_finite(double x) {
  return ((__double2hiint(x) >> 20) & 0x7ff) == 0x7ff;
}

__device__ __forceinline__ bool state_not_finite(const State& s) {
  return not_finite(s.r) | not_finite(s.th) | not_finite(s.ph) | not_finite(s.pr) |
         not_finite(s.pth);
}

// Error test of one component: accept needs |d| <= tol (1 + max(|y|, |o|));
// the ratio (for the step-size controller only) is formed in FP32.
__device__ __forceinline__ void err_component(double y, double o, double d, double tol,
                                              bool& ok, float& err) {
  const double scale = tol * (1.0 + fmax(fabs(y), fabs(o)));
  const double ad = fabs(d);
  ok = ok && (ad <= scale);
  err = fmaxf(err, __fdividef((float)ad, (float)scale));
}

// |x| as FP32 by truncating the significand with integer operations only
// (relative error < 2^-23; values below the FP32 normal range become 0,
// above it +inf). Keeps these conversions off the FP64 pipe.
__device__ __forceinline__ float abs_to_float_rz(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
  const int e = (int)(b >> 52) - 1023 + 127;
  if (e <= 0) return 0.0f;
  if (e >= 255) return __int_as_float(0x7f800000);
  return __int_as_float((e << 23) | (int)((b >> 29) & 0x7fffffull));
}

// The error norm of a step (max over the five components of
// |d| / (tol (1 + max(|y|, |o|)))) in FP32 from truncated copies; the ratio is
// within a relative 1e-6 of the FP64 one. The caller decides accept/reject
// from it and falls back to the exact FP64 test (err_component) only when it
// lies within 1e-5 of 1, so the decision is always the FP64 one.
__device__ __forceinline__ float err_norm32(const State& y, const State& o, const State& d,
                                            float tol32) {
  float err = 0.0f;
#define OSIRIS_ERR32(c)                                                                  \
  err = fmaxf(err, __fdividef(abs_to_float_rz(d.c),                                     \
                              tol32 * (1.0f + fmaxf(abs_to_float_rz(y.c),               \
                                                    abs_to_float_rz(o.c)))))
  OSIRIS_ERR32(r);
  OSIRIS_ERR32(th);
  OSIRIS_ERR32(ph);
  OSIRIS_ERR32(pr);
  OSIRIS_ERR32(pth);
#undef OSIRIS_ERR32
  return err;
}

// Value whose sign tells which side of a stopping surface a state is on;
// the crossing is where it changes sign.
__device__ __forceinline__ double surface_value(int kind, const State& s, double r_cap,
                                                double r_esc) {
  if (kind == SURF_EQUATOR) return (PIO2_HI - s.th) + PIO2_LO;  // sign of cos(theta)
  if (kind == SURF_CAPTURE) return s.r - r_cap;
  return s.r - r_esc;
}

__device__ __forceinline__ bool crosses_equator(const State& y0, const State& y1) {
  const double c0 = (PIO2_HI - y0.th) + PIO2_LO;
  const double c1 = (PIO2_HI - y1.th) + PIO2_LO;
  return (c0 > 0.0 && c1 <= 0.0) || (c0 < 0.0 && c1 >= 0.0);
}

__device__ __forceinline__ const ReqDev* request_of(const KernelArgs& A, int k) {
  return A.reqs ? (A.reqs + k) : &A.single;
}

// Request owning global ray g (largest k with ray_begin <= g).
__device__ __forceinline__ int find_request(const KernelArgs& A, int64_t g) {
  if (A.reqs == nullptr) return 0;
  int lo = 0, hi = A.n_req - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&A.reqs[mid].ray_begin) <= g)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Per-lane totals folded into the stats counters when the lane retires.
struct LaneStats {
  unsigned long long rays = 0, acc = 0, rej = 0, root = 0, rhs = 0, fp64_steps = 0;
  unsigned long long status[6] = {0, 0, 0, 0, 0, 0};
  double max_abs_H = 0.0;
};

__device__ __forceinline__ void flush_stats(const KernelArgs& A, LaneStats& S) {
  if (A.stats == nullptr) return;
  const unsigned FULL = 0xffffffffu;
  unsigned long long v[12] = {S.rays, S.acc, S.rej, S.root, S.rhs, S.status[0], S.status[1],
                              S.status[2], S.status[3], S.status[4], S.status[5], S.fp64_steps};
  double mh = S.max_abs_H;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int q = 0; q < 12; ++q) v[q] += __shfl_xor_sync(FULL, v[q], off);
    mh = fmax(mh, __shfl_xor_sync(FULL, mh, off));
  }
  if ((threadIdx.x & 31) == 0) {
    for (int q = 0; q < 11; ++q)
      if (v[q]) atomicAdd(A.stats + q, v[q]);
    if (v[11]) atomicAdd(A.stats + OSIRIS_STAT_FP64_STEPS, v[11]);
    atomicMax(A.stats + OSIRIS_STAT_MAX_ABS_H, (unsigned long long)__double_as_longlong(mh));
  }
}

}  // namespace osiris_impl
