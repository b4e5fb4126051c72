// The lane state machine shared by the double-float (DF64) and mixed (MIXED)
// trace kernels: a df64 state vector (pairs of FP32, 48-bit significand)
// integrated on the FP32 pipe, with the evaluation of Hamilton's equations
// supplied by a metric policy: double-float for DF64 (trace_df64.cu, stepper
// rk_step_df in step_df.cuh), FP32 for MIXED (trace_mixed.cu, stepper
// rk_step_mixed in step_mixed.cuh). FP64 is used once per ray (initial data,
// the terminal state and the observables) and for the step-length bracket of
// surface location.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "df64.cuh"
#include "rhs_df.cuh"
#include "step_df.cuh"
#include "step_mixed.cuh"
#include "trace_kernel.cuh"

namespace osiris_impl {

__device__ __forceinline__ RayDF to_df(const RayK& K) {
  RayDF k;
  k.a = df_from_double(K.a);
  k.a2 = df_from_double(K.a2);
  k.aE = df_from_double(K.aE);
  k.aL = df_from_double(K.aL);
  k.E = df_from_double(K.E);
  k.L = df_from_double(K.L);
  k.twoE = df_scale(k.E, 2.0f);
  k.twoH0 = 0.0f;
  return k;
}

__device__ __forceinline__ StateDF to_df(const State& s) {
  StateDF d;
  d.r = df_from_double(s.r);
  d.th = df_from_double(s.th);
  d.ph = df_from_double(s.ph);
  d.pr = df_from_double(s.pr);
  d.pth = df_from_double(s.pth);
  return d;
}

__device__ __forceinline__ State to_double(const StateDF& d) {
  State s;
  s.r = df_to_double(d.r);
  s.th = df_to_double(d.th);
  s.ph = df_to_double(d.ph);
  s.pr = df_to_double(d.pr);
  s.pth = df_to_double(d.pth);
  return s;
}

__device__ __forceinline__ RayQDF to_qdf(const RayK& K) {
  RayQDF k;
  k.E = df_from_double(K.E);
  k.L = df_from_double(K.L);
  k.q = df_from_double(K.q);
  k.kap = df_from_double(K.kap);
  k.nq1 = df_from_double(-(1.0 + K.q));
  k.E2 = df_from_double(K.E * K.E);
  k.twoH0 = 0.0f;
  return k;
}

// a < b for normalised df values
__device__ __forceinline__ bool df_lt(df a, df b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}

// Sign of cos(theta) through pi/2 - theta (exact to df64 precision).
__device__ __forceinline__ float df_side(df th) {
  const df t = df_sub(mk(dfc::P1, dfc::P2), th);
  return t.hi != 0.0f ? t.hi : t.lo;
}

// True when any of the values is infinite or NaN: 0 * x is NaN exactly for
// those, and one NaN term makes the sum NaN. One FMA per value on the FP32
// pipe, where a test of the exponent bits takes two or three integer
// instructions and an OR per value.
template <int N>
__device__ __forceinline__ bool any_not_finite(const float (&v)[N]) {
  float z = 0.0f;
#pragma unroll
  for (int i = 0; i < N; ++i) z = fmaf(0.0f, v[i], z);
  return z != z;
}

// The lane state machine of trace_body (trace_kernel.cuh) with a df64 state:
// same modes, same order of tests, same controller; the INTEGRATE path issues
// no FP64 instruction. Surface location keeps its bracket in FP64.
//
// The metric policy Met provides: Ray (its per-ray constants) and ray(K);
// kF32Stages, which stepper integrates (false: rk_step_df with rhs(), the
// double-float evaluation of Hamilton's equations at a df64 point; true:
// rk_step_mixed with rhs_f(), the FP32 evaluation); end_twoH(),
// 2 (H - H0) at the end point in double-float; kTrackH, whether the |H| of
// every step start (from rhs) enters the ray's max |H|; kLocateRel, the
// relative width of the step-length bracket at which surface location stops
// (the resolution of a trial step's end point); kMaxRegs, the register cap.
template <class Met, bool PERSISTENT, int INTEG>
__device__ __forceinline__ void trace_body_df(const KernelArgs& A) {
  const unsigned FULL = 0xffffffffu;
  int mode = MODE_IDLE;
  bool drained = !PERSISTENT;
  LaneStats S;

  RayInfo I;
  typename Met::Ray KD;
  df r_cap, r_esc;
  float tol = 0.0f;
  StateDF y;
  float h = 0.0f, max_abs_H = 0.0f;
  unsigned n_acc = 0, n_rej = 0;
  int kind = 0, side = 0, iters = 0;
  double lo = 0, hi = 0, h_try = 0;  // surface location: the step-length bracket
  df h_try_df = mk(0.0f, 0.0f);       // h_try as the stepper takes it
  float h_step = 0.0f;                // length of the last accepted step
  float flo = 0.0f, fhi = 0.0f;
  StateDF yF, yE;
  std::conditional_t<Met::kF32Stages, LaneCacheF32<INTEG>, LaneCacheDF<INTEG>> LC;

  auto start_ray = [&](int64_t g) {
    State y0;
    if (!load_ray(A, g, I, y0)) return;  // checked build: index check failed
    LC.reset();
    y = to_df(y0);
    KD = Met::ray(I.K);
    KD.twoH0 = (float)(2.0 * I.H0);
    r_cap = df_from_double(I.r_cap);
    r_esc = df_from_double(I.r_esc);
    tol = (float)I.tol;
    h = (float)I.h0;
    max_abs_H = 0.0f;
    n_acc = n_rej = 0;
    mode = MODE_INTEGRATE;
  };

  // The ray has ended with `status` at state fd: keep both and wait (DONE)
  // until complete() writes its outputs together with other lanes' (see
  // complete_finished in trace_kernel.cuh).
  int done_status = 0;
  auto finish = [&](int status, const StateDF& fd) {
    done_status = status;
    yF = fd;
    mode = MODE_DONE;
  };

  // The end-point |H| check and the outputs of a DONE lane; retires it. The
  // check evaluates 2 (H - H0) at the final state with the double-float
  // equations (error ~2^-48 of the terms of 2H), on the FP32 pipe; only the
  // outputs are formed in FP64.
  auto complete = [&]() {
    const State f = to_double(yF);
    float mh = max_abs_H;
    if (done_status != OSIRIS_STATUS_ERROR) {
      mh = fmaxf(mh, fabsf(0.5f * Met::end_twoH(KD, I.K, yF)));
      S.rhs += 1;
    }
    write_outputs(A, I, done_status, f, (double)mh, n_acc, n_rej, S);
    mode = MODE_IDLE;
  };

  // Signed distance to the surface (pi/2 - theta, r - r_cap or r - r_esc),
  // formed in double-float (the difference of nearby values is exact) and
  // rounded to FP32: its sign and its size relative to the tolerance are all
  // surface location needs, so no FP64 instruction is spent on it.
  auto surf = [&](int k, const StateDF& s) -> float {
    const df d = (k == SURF_EQUATOR) ? df_sub(mk(dfc::P1, dfc::P2), s.th)
                                     : df_sub(s.r, k == SURF_CAPTURE ? r_cap : r_esc);
    return __fadd_rn(d.hi, d.lo);
  };

  // Next trial step length of the bracket [lo, hi]: the regula falsi point
  // lo + (hi - lo) t, t = f_lo / (f_lo - f_hi) in FP32 (f_lo, f_hi have
  // opposite signs, so t is in (0, 1) without cancellation); the midpoint if
  // rounding put it on an end.
  auto next_trial = [&]() {
    const float t = __fdividef(flo, __fsub_rn(flo, fhi));
    h_try = fma(hi - lo, (double)t, lo);
    if (!(h_try > lo && h_try < hi)) h_try = 0.5 * (lo + hi);
    h_try_df = df_from_double(h_try);
  };

  auto begin_locate = [&](int k, float hs, const StateDF& o) {
    kind = k;
    lo = 0.0;
    hi = hs;
    flo = surf(k, y);
    fhi = surf(k, o);
    yF = o;
    side = 0;
    iters = 0;
    next_trial();
    mode = MODE_LOCATE;
  };

  // `fresh`: the last attempt was the accepted step itself.
  auto after_accept = [&](float hs, const StateDF& o, bool fresh) {
    if (df_lt(o.r, r_cap)) {
      begin_locate(SURF_CAPTURE, hs, o);
    } else if (df_lt(r_esc, o.r)) {
      begin_locate(SURF_ESCAPE, hs, o);
    } else {
      y = o;
      if (fresh)
        LC.accepted();
      else
        LC.reset();
      mode = MODE_INTEGRATE;
      if ((int64_t)(n_acc + n_rej) >= I.max_steps) finish(OSIRIS_STATUS_MAXSTEP, y);
    }
  };

  init_claim<PERSISTENT>(A);

  for (;;) {
    if (complete_finished(A, mode)) complete();
    const bool busy = (mode == MODE_INTEGRATE) || (mode == MODE_LOCATE);
    if (mode == MODE_IDLE) {
      const int64_t g = next_claimed(A);
      if (g >= 0) start_ray(g);
    }
    if (PERSISTENT) {
      int64_t first = 0;
      const int got = refill(A, (mode == MODE_IDLE) && !drained, busy, first);
      if (got > 0) {
        set_claim(first + 1, got - 1);
        start_ray(first);
      } else if (got < 0) {
        drained = true;
      }
    }
    if (!__any_sync(FULL, mode != MODE_IDLE || has_claim())) break;
    if (mode != MODE_INTEGRATE && mode != MODE_LOCATE) continue;

    const float hs_f = fminf(h, 0.1f * y.r.hi);
    // the step length: no FP64 instruction on the integration path
    const df hd = (mode == MODE_LOCATE) ? h_try_df : mk(hs_f, 0.0f);
    StateDF o;
    float d[5];
    float twoH;
    if constexpr (Met::kF32Stages)
      rk_step_mixed<Met, INTEG>(KD, LC, y, hd, o, d, twoH);
    else
      rk_step_df<Met, INTEG>(KD, LC, y, hd, o, d, twoH);
    S.rhs += 6;

    if (mode == MODE_INTEGRATE) {
      if (Met::kTrackH) max_abs_H = fmaxf(max_abs_H, fabsf(0.5f * twoH));  // 2 (H - H0) at y
      const float ys[5] = {y.r.hi, y.th.hi, y.ph.hi, y.pr.hi, y.pth.hi};
      const float os[5] = {o.r.hi, o.th.hi, o.ph.hi, o.pr.hi, o.pth.hi};
      const float od[10] = {os[0], os[1], os[2], os[3], os[4], d[0], d[1], d[2], d[3], d[4]};
      const bool bad = any_not_finite(od);
      bool ok = true;
      float err = 0.0f;
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const float scale = tol * (1.0f + fmaxf(fabsf(ys[c]), fabsf(os[c])));
        const float ad = fabsf(d[c]);
        ok = ok && (ad <= scale);
        err = fmaxf(err, __fdividef(ad, scale));
      }
      if (bad) {
        finish(OSIRIS_STATUS_ERROR, y);
        continue;
      }
      if (ok) {
        ++n_acc;
        const float grow = fminf(5.0f, fmaxf(0.2f, 0.9f * exp2f(-0.2f * log2f(err))));
        h = hs_f * grow;
        h_step = hs_f;
        yE = o;
        if (I.disk && ((df_side(y.th) > 0.0f && df_side(o.th) <= 0.0f) ||
                       (df_side(y.th) < 0.0f && df_side(o.th) >= 0.0f)))
          begin_locate(SURF_EQUATOR, h_step, o);
        else
          after_accept(h_step, o, true);
      } else {
        ++n_rej;
        const float shrink = fmaxf(0.1f, 0.9f * exp2f(-0.25f * log2f(err)));
        h = hs_f * shrink;
        if ((int64_t)(n_acc + n_rej) >= I.max_steps) finish(OSIRIS_STATUS_MAXSTEP, y);
      }
    } else {  // MODE_LOCATE: Illinois-modified regula falsi on the step length
      S.root += 1;
      ++iters;
      const float os[5] = {o.r.hi, o.th.hi, o.ph.hi, o.pr.hi, o.pth.hi};
      if (any_not_finite(os)) {
        finish(OSIRIS_STATUS_ERROR, y);
        continue;
      }
      const double hs = h_try;
      const float f = surf(kind, o);
      const bool to_lo = (f != 0.0f) && ((f > 0.0f) == (flo > 0.0f));
      if (to_lo) {
        lo = hs;
        flo = f;
        if (side == -1) fhi *= 0.5f;
        side = -1;
      } else {
        hi = hs;
        fhi = f;
        yF = o;
        if (side == +1) flo *= 0.5f;
        side = +1;
      }
      const float ftol = (kind == SURF_EQUATOR)
                             ? 1e-15f
                             : 1e-14f * (kind == SURF_CAPTURE ? r_cap.hi : r_esc.hi);
      const bool done = (f == 0.0f) || (!to_lo && fabsf(f) <= ftol) ||
                        (hi - lo <= Met::kLocateRel * hi) || iters >= 64;
      if (!done) {
        next_trial();
      } else if (kind == SURF_CAPTURE) {
        finish(OSIRIS_STATUS_CAPTURED, yF);
      } else if (kind == SURF_ESCAPE) {
        finish(OSIRIS_STATUS_ESCAPED, yF);
      } else {
        const double rx = df_to_double(yF.r);
        if (rx >= I.r_in && rx <= I.r_out)
          finish(OSIRIS_STATUS_DISK, yF);
        else
          after_accept(h_step, yE, false);
      }
    }
  }
  flush_stats(A, S);
}

}  // namespace osiris_impl
