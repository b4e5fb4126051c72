// Mixed-precision trace kernels (OSIRIS_MIXED), Kerr and the q-metric: the
// lane state machine of the DF64 kernels (trace_df_body.cuh) with the six
// evaluations of Hamilton's equations of every attempt in FP32 (rhs_f32.cuh)
// and a stepper that sums their derivatives in FP32 (step_mixed.cuh). The
// state and the stage inputs keep df64 precision (FP32 with compensated
// sums), so adding a small increment to the state loses nothing; the
// derivatives carry FP32 rounding, ~1e-7 of |k|, and the sums over stages
// (increments, error estimate) add roundings of the same relative size. No
// step of the integration runs on the FP64 pipe: FP64 only sets up each ray,
// keeps the step-length bracket of surface location and forms the outputs.
//
// Tolerance range. The embedded error estimate h sum_s (b_s - b*_s)(k_s - k_1)
// then carries a noise of ~1e-8 h |k| ~ 1e-8 (h/tau) |y| (tau: time scale of
// the solution), against the local error tol (1 + |y|) that the controller
// compares it with. At tol 1e-8 the accepted steps have h/tau ~ 0.03 and the
// noise is a few percent of the estimate; at 1e-10 it is as large as the
// estimate and the controller would shrink the steps to chase it. MIXED is
// meant for tolerances of 1e-8 and looser; DF64 covers the tighter ones.
//
// |H|. The FP32 evaluations' own 2H carries the rounding of its largest terms
// (P^2 / Delta grows without bound towards the horizon), so it does not track
// the constraint; a ray's |H| output is that of its end point, evaluated in
// double-float (rhs_df) as in the DF64 kernels.
//
// Surface location. A trial step's end point carries the FP32 rounding of its
// stage derivatives, ~1e-7 h |k|, so the step-length bracket is resolved to a
// relative width of 2e-7, not to the DF64 kernels' 4e-16.
#include <cuda_runtime.h>

#include "rhs_f32.cuh"
#include "trace_df_body.cuh"

namespace osiris_impl {

// Registers capped so that more blocks of 128 threads are resident per SM
// than the code's natural ~190 registers allow: the FP32 stepper keeps only
// the df64 state, the stage inputs and FP32 sums live, and the extra warps
// hide more of the dependent FP32 chains than the added spills (L1 hits)
// cost. Measured on the 12 x 1024^2 Kerr set at tol 1e-8 (Mrays/s, Cash-Karp,
// refill at 32 idle lanes): 96 registers 160.9, 80 (6 blocks): 162.3, 72:
// 154.7, 64: 153.0; on the six q-metric renders: 80: 117.6, 72: 118.9, 64:
// 123.3, 56 (9 blocks): 127.1.
#ifndef OSIRIS_MIXED_MAXREGS
#define OSIRIS_MIXED_MAXREGS 80
#endif
#ifndef OSIRIS_MIXED_Q_MAXREGS
#define OSIRIS_MIXED_Q_MAXREGS 56
#endif

struct KerrMixed {
  using Ray = RayF32;
  static constexpr int kMaxRegs = OSIRIS_MIXED_MAXREGS;
  static constexpr bool kTrackH = false;
  static constexpr bool kF32Stages = true;
  static constexpr double kLocateRel = 2e-7;
  static __device__ __forceinline__ Ray ray(const RayK& K) {
    Ray k;
    k.a = (float)K.a;
    k.a2 = (float)K.a2;
    k.aE = (float)K.aE;
    k.aL = (float)K.aL;
    k.E = (float)K.E;
    k.L = (float)K.L;
    k.twoE = (float)(2.0 * K.E);
    const double sq = sqrt(fmax(0.0, 1.0 - K.a2));
    k.rp = df_from_double(1.0 + sq);
    k.rm = (float)(1.0 - sq);
    k.twoH0 = 0.0f;
    return k;
  }
  static __device__ __forceinline__ void rhs_f(const Ray& K, const PointF32& x, float& dr,
                                               float& dth, float& dph, float& dpr, float& dpth,
                                               float& twoH) {
    rhs_f32(K, x, dr, dth, dph, dpr, dpth, twoH);
  }
  // 2 (H - H0) at the end point with the double-float equations of DF64.
  static __device__ __forceinline__ float end_twoH(const Ray& KD, const RayK& K,
                                                   const StateDF& y) {
    RayDF k = to_df(K);
    k.twoH0 = KD.twoH0;
    df dr, dth, dph, dpr, dpth;
    float twoH;
    rhs_df(k, y.r, y.th, y.pr, y.pth, dr, dth, dph, dpr, dpth, twoH);
    return twoH;
  }
};

// The q-metric (Appendix A) with the same stepper; its end-point |H| from
// the double-float q-metric equations (rhs_q_df).
struct QMetricMixed {
  using Ray = RayQF32;
  static constexpr int kMaxRegs = OSIRIS_MIXED_Q_MAXREGS;
  static constexpr bool kTrackH = false;
  static constexpr bool kF32Stages = true;
  static constexpr double kLocateRel = 2e-7;
  static __device__ __forceinline__ Ray ray(const RayK& K) {
    Ray k;
    k.E = (float)K.E;
    k.L = (float)K.L;
    k.q = (float)K.q;
    k.kap = (float)K.kap;
    k.nq1 = (float)(-(1.0 + K.q));
    k.E2 = (float)(K.E * K.E);
    k.twoH0 = 0.0f;
    return k;
  }
  static __device__ __forceinline__ void rhs_f(const Ray& K, const PointF32& x, float& dr,
                                               float& dth, float& dph, float& dpr, float& dpth,
                                               float& twoH) {
    rhs_q_f32(K, x, dr, dth, dph, dpr, dpth, twoH);
  }
  static __device__ __forceinline__ float end_twoH(const Ray& KD, const RayK& K,
                                                   const StateDF& y) {
    RayQDF k = to_qdf(K);
    k.twoH0 = KD.twoH0;
    df dr, dth, dph, dpr, dpth;
    float twoH;
    rhs_q_df(k, y.r, y.th, y.pr, y.pth, dr, dth, dph, dpr, dpth, twoH);
    return twoH;
  }
};

template <class Met, int INTEG>
__global__ void __maxnreg__(Met::kMaxRegs) trace_mixed_plain(const __grid_constant__ KernelArgs A) {
  trace_body_df<Met, false, INTEG>(A);
}

template <class Met, int INTEG>
__global__ void __maxnreg__(Met::kMaxRegs)
    trace_mixed_persistent(const __grid_constant__ KernelArgs A) {
  trace_body_df<Met, true, INTEG>(A);
}

template <class Met, int INTEG>
static const void* mixed_kernel(Kernel kind) {
  return kind == Kernel::kPersistent ? (const void*)trace_mixed_persistent<Met, INTEG>
                                     : (const void*)trace_mixed_plain<Met, INTEG>;
}

template <class Met>
static const void* mixed_kernel(Kernel kind, int integrator) {
  return integrator == OSIRIS_RKDP45 ? mixed_kernel<Met, OSIRIS_RKDP45>(kind)
                                     : mixed_kernel<Met, OSIRIS_RKCK45>(kind);
}

static const void* select_mixed(Kernel kind, int integrator, int spacetime) {
  return spacetime == OSIRIS_SPACETIME_QMETRIC ? mixed_kernel<QMetricMixed>(kind, integrator)
                                               : mixed_kernel<KerrMixed>(kind, integrator);
}

int launch_trace_mixed(const KernelArgs& args, Kernel kind, int integrator, int grid, int block,
                       void* stream) {
  const int spacetime = args.reqs ? args.spacetime : args.single.spacetime;
  void* params[] = {const_cast<KernelArgs*>(&args)};
  return (int)cudaLaunchKernel(select_mixed(kind, integrator, spacetime), dim3(grid),
                               dim3(block), params, 0, static_cast<cudaStream_t>(stream));
}

int occupancy_mixed(Kernel kind, int integrator, int spacetime, int block, int* blocks_per_sm) {
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      blocks_per_sm, select_mixed(kind, integrator, spacetime), block, 0);
}

}  // namespace osiris_impl
