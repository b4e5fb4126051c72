// The trace kernel: one ray per lane, uniform Cash-Karp attempts, stopping
// surfaces located inside the step, per-ray epilogue, and (persistent grids)
// lane refill from a device ray queue. Instantiated per precision by
// trace_fp64.cu and trace_mixed.cu through the Stepper policy:
//   Stepper::RayCache                         per-ray data the stepper derives
//   Stepper::prepare(K, cache)                once per ray
//   Stepper::LaneCache                        stage values carried between attempts
//                                             (first same as last)
//   Stepper::reset(lane)                      the state changed other than by a step
//   Stepper::accepted(lane)                   y <- o after an accepted attempt
//   Stepper::attempt(K, cache, lane, y, h, o, d, twoH) -> one embedded RK attempt
//   Stepper::twoH(K, y)                       -> 2H at a state (FP64)
#pragma once

#include "checked.cuh"
#include "trace_device.cuh"

namespace osiris_impl {

// Per-ray identity and constants, common to every lane state machine.
struct RayInfo {
  int req;
  int64_t local;  // index of the ray inside its request
  RayK K;
  double H0;      // mass shell: the error tracked is |H - H0| (Sec. 3.1)
  double r_cap, r_esc, r_in, r_out, tol, h0;
  int disk;
  int64_t max_steps;
};

#ifdef OSIRIS_CHECKED
// Count a failed index check in the caller's stats (checked build only).
__device__ __forceinline__ void record_check_failure(const KernelArgs& A, unsigned code,
                                                     int64_t g) {
  if (A.stats == nullptr) return;
  atomicAdd(A.stats + OSIRIS_STAT_CHECK_FAILS, 1ull);
  atomicMax(A.stats + OSIRIS_STAT_CHECK_WORST, check_word(code, g));
}
#endif

// Ray g of the launch: its request, constants and initial state (Sec. 2.3,
// Eq. momentums: pixel centre -> p_theta, L, E, p_r at t = 0, r = r0,
// theta = theta0, phi = 0; or explicit initial data for the test hook).
// Returns false (checked build only) when an index check fails: nothing of
// the ray has been read and the lane must not start it.
__device__ __forceinline__ bool load_ray(const KernelArgs& A, int64_t g, RayInfo& I, State& y) {
  I.req = find_request(A, g);
#ifdef OSIRIS_CHECKED
  if (const unsigned code = check_ray_request(g, A.total_rays, I.req, A.reqs ? A.n_req : 1)) {
    record_check_failure(A, code, g);
    return false;
  }
#endif
  const ReqDev* R = request_of(A, I.req);
  I.local = g - R->ray_begin + R->pixel_offset;
#ifdef OSIRIS_CHECKED
  const int64_t limit =
      R->explicit_states ? R->pixel_offset + R->n_rays : (int64_t)R->nx * (int64_t)R->ny;
  if (const unsigned code = check_ray_pixel(g, R->ray_begin, R->n_rays, I.local, limit)) {
    record_check_failure(A, code, g);
    return false;
  }
#endif
  const double a = R->a;
  I.K.a = a;
  I.K.a2 = a * a;
  I.K.q = R->q;
  I.K.kap = R->q * (2.0 + R->q);
  I.H0 = R->H0;
  if (R->explicit_states) {
    const double* st = R->states + 6 * I.local;
    y.r = st[1];
    y.th = st[2];
    y.ph = st[3];
    y.pr = st[4];
    y.pth = st[5];
    I.K.E = R->E[I.local];
    I.K.L = R->L[I.local];
  } else {
    const int64_t i = I.local % R->nx, j = I.local / R->nx;
    const double x = R->x_min + ((double)i + 0.5) * R->x_span / R->nx;
    const double yy = R->y_min + ((double)j + 0.5) * R->y_span / R->ny;
    const double Pth = yy / R->r0, Pph = -x / R->r0;
    I.K.E = R->inv_At + x * R->e_x;
    I.K.L = x * R->l_x;
    y.r = R->r0;
    y.th = R->th0;
    y.ph = 0.0;
    y.pth = yy * R->pth_y;
    y.pr = -sqrt(R->grr * (1.0 - Pth * Pth - Pph * Pph));
  }
  I.K.aE = a * I.K.E;
  I.K.aL = a * I.K.L;
  I.K.E2 = I.K.E + I.K.E;
  I.r_cap = R->r_cap;
  I.r_esc = R->r_esc;
  I.r_in = R->r_in;
  I.r_out = R->r_out;
  I.disk = R->disk;
  I.tol = R->tol;
  I.max_steps = R->max_steps;
  I.h0 = R->h0;
  return true;
}

// x reduced into [0, 2 pi): x - 2 pi floor(x / (2 pi)) with one rounding in
// the fused multiply-add (error a few ulp of x), then the ends fixed.
__device__ __forceinline__ double wrap_2pi(double x) {
  constexpr double INV_TWO_PI = 0.15915494309189535;
  double t = fma(-TWO_PI, floor(x * INV_TWO_PI), x);
  if (t < 0.0) t += TWO_PI;
  if (t >= TWO_PI) t -= TWO_PI;
  return t;
}

// Write the outputs of a finished ray (terminal state f, final max |H|) and
// fold it into the lane's counters.
__device__ __forceinline__ void write_outputs(const KernelArgs& A, const RayInfo& I, int status,
                                              const State& f, double max_abs_H, unsigned n_acc,
                                              unsigned n_rej, LaneStats& S) {
  const ReqDev* R = request_of(A, I.req);
  const int64_t local = I.local;
  const osiris_outputs& O = R->out;
  if (O.status) O.status[local] = (uint8_t)status;
  if (O.r) O.r[local] = f.r;
  if (O.theta) O.theta[local] = f.th;
  if (O.phi) O.phi[local] = f.ph;
  if (O.max_abs_H) O.max_abs_H[local] = max_abs_H;
  if (O.steps) O.steps[local] = n_acc;
  int ci = -1, cj = -1, par = 0;
  if (status == OSIRIS_STATUS_ESCAPED) {
    // celestial checkerboard: fold theta into [0, pi], wrap phi into [0, 2pi)
    // (angles reduced by floor instead of the library fmod, cells by the
    // host's reciprocal of the cell size: a cell index can differ from the
    // divided one only within ~1e-15 rad of an edge)
    double t = wrap_2pi(f.th);
    double p = f.ph;
    if (t > PI_D) {
      t = TWO_PI - t;
      p += PI_D;
    }
    const double q = wrap_2pi(p + R->phase_rad);
    ci = (int)floor(t * R->inv_cell);
    cj = (int)floor(q * R->inv_cell);
    ci = min(max(ci, 0), R->n_th_cells - 1);
    cj = ((cj % R->n_ph_cells) + R->n_ph_cells) % R->n_ph_cells;
    par = (ci + cj) & 1;
  }
  if (O.cell_i) O.cell_i[local] = (int16_t)ci;
  if (O.cell_j) O.cell_j[local] = (int16_t)cj;
  if (O.parity) O.parity[local] = (uint8_t)par;
  double g = 0.0, Iobs = 0.0, rh = 0.0;
  if (status == OSIRIS_STATUS_DISK) {
    // Disk gas on circular orbits (Sec. 5): Keplerian Omega = 1/(r^3/2 + a),
    // or constant l0 = -u_phi/u_t: Omega = -(g_tphi + l0 g_tt)/(g_phph + l0 g_tphi).
    // u^t from the normalisation g_ab u^a u^b = -1 in the equatorial plane;
    // g = 1/(u^t (E - Omega L)); I = g^3 / r^2 (0 where no timelike orbit exists).
    const double r = f.r, a = I.K.a;
    const double gtt = -(1.0 - 2.0 / r);
    const double gtp = -2.0 * a / r;
    const double gpp = r * r + a * a + 2.0 * a * a / r;
    const double Om = (R->disk == OSIRIS_DISK_CONSTANT_L)
                          ? -(gtp + R->l0 * gtt) / (gpp + R->l0 * gtp)
                          : 1.0 / fma(r, sqrt(r), a);
    const double norm = -gtt - 2.0 * Om * gtp - Om * Om * gpp;
    if (norm > 0.0) {
      g = sqrt(norm) / (I.K.E - Om * I.K.L);
      Iobs = g * g * g / (r * r);
    }
    rh = r;
  }
  if (O.g) O.g[local] = g;
  if (O.intensity) O.intensity[local] = Iobs;
  if (O.r_hit) O.r_hit[local] = rh;
  S.rays += 1;
  S.status[status] += 1;
  S.acc += n_acc;
  S.rej += n_rej;
  // a ray that ended on a non-finite state may have tracked an infinite |H|
  if (status != OSIRIS_STATUS_ERROR) S.max_abs_H = fmax(S.max_abs_H, max_abs_H);
}

// Take the next rays of a persistent grid from the device queue for the lanes
// that need one: one atomic per warp claims rays_per_lane consecutive rays
// for each such lane. A warp with busy lanes refills only when at least
// refill_lanes of its lanes need rays (a warp with no busy lane always
// refills, so no warp waits forever). Returns the number of rays claimed by
// this lane (their first index in `first`), 0 when it claimed none this time,
// or -1 when the queue is drained.
__device__ __forceinline__ int refill(const KernelArgs& A, bool need, bool busy,
                                      int64_t& first) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned m = __ballot_sync(FULL, need);
  const unsigned b = __ballot_sync(FULL, busy);
  if (!m || (b && __popc(m) < A.refill_lanes)) return 0;
  const int leader = __ffs(m) - 1;
  const unsigned long long per = (unsigned long long)A.rays_per_lane;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(A.queue, (unsigned long long)__popc(m) * per);
  base = __shfl_sync(FULL, base, leader);
  if (!need) return 0;
  const unsigned long long g = base + __popc(m & ((1u << lane) - 1u)) * per;
  const unsigned long long total = (unsigned long long)A.total_rays;
  if (g >= total) return -1;
  first = (int64_t)g;
  return (int)(total - g < per ? total - g : per);
}

// Lanes whose ray has ended (DONE) complete it (end-point check, outputs)
// together: once refill_lanes of the warp are DONE, or when no lane of the
// warp is still integrating. Their warp instructions, FP64 for the most part,
// are then shared by several lanes instead of being issued for one lane at a
// time as each ray ends. Warp-uniform decision; returns true for the lanes
// that complete now.
__device__ __forceinline__ bool complete_finished(const KernelArgs& A, int mode) {
  const unsigned FULL = 0xffffffffu;
  const unsigned done = __ballot_sync(FULL, mode == MODE_DONE);
  if (!done) return false;
  const unsigned busy = __ballot_sync(FULL, mode == MODE_INTEGRATE || mode == MODE_LOCATE);
  return (mode == MODE_DONE) && (!busy || __popc(done) >= A.refill_lanes);
}

// Rays a lane has claimed and not yet started, [next, end), one slot per
// thread of the block (at most 256). They live in shared memory, and are
// read and written only by the lane itself when it is idle, so no register
// holds them across the attempt loop. Volatile: the accesses stay in memory.
constexpr int kClaimSlots = 256;

struct LaneClaims {
  volatile long long next[kClaimSlots], end[kClaimSlots];
};

__device__ __forceinline__ LaneClaims& lane_claims() {
  __shared__ LaneClaims claims;
  return claims;
}

// The lane's first claim: a plain launch (one launch thread per ray range)
// gives each thread rays_per_lane consecutive rays from thread index x
// rays_per_lane; a persistent grid starts with none and refills.
template <bool PERSISTENT>
__device__ __forceinline__ void init_claim(const KernelArgs& A) {
  LaneClaims& C = lane_claims();
  long long next = 0, end = 0;
  if (!PERSISTENT) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    next = t * A.rays_per_lane;
    end = next + A.rays_per_lane;
    if (end > A.total_rays) end = A.total_rays;
  }
  C.next[threadIdx.x] = next;
  C.end[threadIdx.x] = end;
}

// Next claimed ray of an idle lane (-1 when its claim is used up).
__device__ __forceinline__ int64_t next_claimed(const KernelArgs&) {
  LaneClaims& C = lane_claims();
  const long long g = C.next[threadIdx.x];
  if (g >= C.end[threadIdx.x]) return -1;
  C.next[threadIdx.x] = g + 1;
  return g;
}

// True when the lane still holds claimed rays (idle lanes only ask).
__device__ __forceinline__ bool has_claim() {
  LaneClaims& C = lane_claims();
  return C.next[threadIdx.x] < C.end[threadIdx.x];
}

__device__ __forceinline__ void set_claim(int64_t first, int count) {
  LaneClaims& C = lane_claims();
  C.next[threadIdx.x] = first;
  C.end[threadIdx.x] = first + count;
}

template <class Stepper, bool PERSISTENT>
__device__ __forceinline__ void trace_body(const KernelArgs& A) {
  const unsigned FULL = 0xffffffffu;
  if (Stepper::kTrigTable) trig_table_init();
  if (Stepper::kExpLogTable) explog_table_init();

  int mode = MODE_IDLE;
  bool drained = !PERSISTENT;
  LaneStats S;

  // ray identity and constants
  RayInfo I;
  RayK& K = I.K;
  typename Stepper::RayCache RC;
  typename Stepper::LaneCache LC;
  double& r_cap = I.r_cap;
  double& r_esc = I.r_esc;
  double& r_in = I.r_in;
  double& r_out = I.r_out;
  double& tol = I.tol;
  int& disk = I.disk;
  int64_t& max_steps = I.max_steps;
  // integration state
  State y;
  float tol32 = 0.0f;
  double h = 0;
  long long max_abs_H = 0;  // bit pattern of max |H - H0| (non-negative doubles order as integers)
  unsigned n_acc = 0, n_rej = 0;
  // surface location (LOCATE)
  int kind = 0, side = 0, iters = 0;
  double lo = 0, hi = 0, flo = 0, fhi = 0, h_try = 0, h_step = 0;
  State yF, yE;  // state at the upper bracket end; end of the accepted step

  auto start_ray = [&](int64_t g) {
    if (!load_ray(A, g, I, y)) return;  // checked build: index check failed
    tol32 = (float)I.tol;
    Stepper::prepare(K, RC);
    Stepper::reset(LC);
    h = I.h0;
    max_abs_H = 0;
    n_acc = n_rej = 0;
    mode = MODE_INTEGRATE;
  };

  // The ray has ended with `status` at state f: keep both and wait (DONE)
  // until complete() writes its outputs together with other lanes' (see
  // complete_finished).
  int done_status = 0;
  auto finish = [&](int status, const State& f) {
    done_status = status;
    yF = f;
    mode = MODE_DONE;
  };

  // The end-point |H| check and the outputs of a DONE lane; retires it.
  auto complete = [&]() {
    if (done_status != OSIRIS_STATUS_ERROR) {
      track_abs_H(max_abs_H, Stepper::twoH(K, yF), I.H0);
      S.rhs += 1;
    }
    write_outputs(A, I, done_status, yF, __longlong_as_double(max_abs_H), n_acc, n_rej, S);
    mode = MODE_IDLE;
  };

  // Start locating the crossing of `surf` inside the accepted step y -> o.
  auto begin_locate = [&](int surf, double hs, const State& o) {
    kind = surf;
    lo = 0.0;
    hi = hs;
    flo = surface_value(surf, y, r_cap, r_esc);
    fhi = surface_value(surf, o, r_cap, r_esc);
    yF = o;
    side = 0;
    iters = 0;
    h_try = (lo * fhi - hi * flo) / (fhi - flo);
    if (!(h_try > lo && h_try < hi)) h_try = 0.5 * (lo + hi);
    mode = MODE_LOCATE;
  };

  // After an accepted step without a disk hit: capture and escape tests on
  // the step end o (in this order), else continue from o. `fresh`: the last
  // attempt was the accepted step itself (its end-stage values are current).
  auto after_accept = [&](double hs, const State& o, bool fresh) {
    if (o.r < r_cap) {
      begin_locate(SURF_CAPTURE, hs, o);
    } else if (o.r > r_esc) {
      begin_locate(SURF_ESCAPE, hs, o);
    } else {
      y = o;
      if (fresh)
        Stepper::accepted(LC);
      else
        Stepper::reset(LC);
      mode = MODE_INTEGRATE;
      if ((int64_t)(n_acc + n_rej) >= max_steps) finish(OSIRIS_STATUS_MAXSTEP, y);
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

    const double hs = (mode == MODE_LOCATE) ? h_try : fmin(h, 0.1 * y.r);
    State o, d;
    double twoH;
    const bool fp64_step = Stepper::attempt(K, RC, LC, y, hs, o, d, twoH);
    S.rhs += 6;
    S.fp64_steps += fp64_step ? 1 : 0;

    if (mode == MODE_INTEGRATE) {
      track_abs_H(max_abs_H, twoH, I.H0);
      if (state_not_finite(o) || state_not_finite(d)) {
        finish(OSIRIS_STATUS_ERROR, y);
        continue;
      }
      float err = err_norm32(y, o, d, tol32);
      bool ok = err < 1.0f;
      if (fabsf(err - 1.0f) < 1e-5f) {  // too close to call in FP32: exact FP64 test
        ok = true;
        err = 0.0f;
        err_component(y.r, o.r, d.r, tol, ok, err);
        err_component(y.th, o.th, d.th, tol, ok, err);
        err_component(y.ph, o.ph, d.ph, tol, ok, err);
        err_component(y.pr, o.pr, d.pr, tol, ok, err);
        err_component(y.pth, o.pth, d.pth, tol, ok, err);
      }
      if (ok) {
        ++n_acc;
        // step-size controller (FP32 is enough to size the next step):
        // min(5, max(0.2, 0.9 err^-1/5))
        const float grow = fminf(5.0f, fmaxf(0.2f, 0.9f * exp2f(-0.2f * log2f(err))));
        h = hs * float_to_double(grow);
        h_step = hs;
        yE = o;
        if (disk && crosses_equator(y, o))
          begin_locate(SURF_EQUATOR, hs, o);
        else
          after_accept(hs, o, true);
      } else {
        ++n_rej;
        const float shrink = fmaxf(0.1f, 0.9f * exp2f(-0.25f * log2f(err)));
        h = hs * float_to_double(shrink);
        if ((int64_t)(n_acc + n_rej) >= max_steps) finish(OSIRIS_STATUS_MAXSTEP, y);
      }
    } else {  // MODE_LOCATE: Illinois-modified regula falsi on the step length
      S.root += 1;
      ++iters;
      if (state_not_finite(o)) {
        finish(OSIRIS_STATUS_ERROR, y);
        continue;
      }
      const double f = surface_value(kind, o, r_cap, r_esc);
      const bool to_lo = (f != 0.0) && ((f > 0.0) == (flo > 0.0));
      if (to_lo) {
        lo = hs;
        flo = f;
        if (side == -1) fhi *= 0.5;
        side = -1;
      } else {
        hi = hs;
        fhi = f;
        yF = o;
        if (side == +1) flo *= 0.5;
        side = +1;
      }
      const double ftol = (kind == SURF_EQUATOR) ? 1e-15 : 1e-14 * (kind == SURF_CAPTURE ? r_cap : r_esc);
      // Stepper::kLocateRel: the relative bracket width below which the
      // stepper's own rounding noise decides the sign of f (0 for FP64)
      const bool done = (f == 0.0) || (!to_lo && fabs(f) <= ftol) ||
                        (hi - lo <= (4e-16 + Stepper::kLocateRel) * hi) || iters >= 64;
      if (!done) {
        h_try = (lo * fhi - hi * flo) / (fhi - flo);
        if (!(h_try > lo && h_try < hi)) h_try = 0.5 * (lo + hi);
      } else if (kind == SURF_CAPTURE) {
        finish(OSIRIS_STATUS_CAPTURED, yF);
      } else if (kind == SURF_ESCAPE) {
        finish(OSIRIS_STATUS_ESCAPED, yF);
      } else if (yF.r >= r_in && yF.r <= r_out) {
        finish(OSIRIS_STATUS_DISK, yF);
      } else {
        // equatorial crossing outside the disk: the accepted step stands;
        // run the capture / escape tests on its end point
        after_accept(h_step, yE, false);
      }
    }
  }
  flush_stats(A, S);
}

}  // namespace osiris_impl
