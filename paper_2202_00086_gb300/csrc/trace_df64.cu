// Double-float trace kernels. Every Cash-Karp attempt of the integration runs
// in df64 arithmetic (pairs of FP32, 48-bit significand) on the FP32 pipe,
// which on GB300 is ~70x the FP64 pipe: the six evaluations of Hamilton's
// equations, the stage sums, the increment, the error estimate, the error
// test, the stopping-surface tests and the end-point |H|. The state between
// steps is a df64 vector too. FP64 is used only once per ray (initial data,
// the terminal state and the observables) and for the step-length bracket of
// surface location.
//
// Stage sums. With d_j = k_j - k_1 (j >= 2), the Cash-Karp combinations are
//   stage input  y_i = y + c_i h k_1 + h sum_j a_ij d_j      (sum_j a_ij = c_i)
//   increment        = h k_1 + h sum_i b_i d_i                (sum_i b_i = 1)
//   error estimate   = h sum_i (b_i - b*_i) d_i               (sum = 0)
// The increment is formed in df64 with df64 weights. The error estimate
// cancels to O(h^5), but every d_i is exact to df64 precision, so the leading
// words summed in FP32 keep its relative error near 2^-24 (h/T)^-3 / 30 (T:
// time scale of the solution), a fraction of a percent at tol 1e-10 (the
// derivation is at rk_step_df). In a stage input the part h sum_j a_ij d_j
// is O(h/T) smaller than the stage's step and reaches the result only
// through one more factor h/T, so it is summed in FP32 too.
//
// The six stages run as a loop with one copy of the evaluation of Hamilton's
// equations (six inlined df64 copies overflow the instruction cache), and
// every stage sum is kept in registers.
//
// The evaluations (Kerr and q-metric) are in rhs_df.cuh, the attempt and its
// tableaus in step_df.cuh, the lane state machine in trace_df_body.cuh; this
// file holds the double-float metric policies and the launchers.
#include "trace_df_body.cuh"

namespace osiris_impl {

// Metric policies of the double-float kernels: the ray constants, the
// evaluation, and the register cap.
// Registers capped at 128 so that four blocks of 128 threads (16 warps) are
// resident per SM: the double-float dependency chains need the extra warps
// more than they lose to the spilled values, which stay in L1 as long as no
// shared memory is reserved. Measured on the 12 x 1024^2 Kerr set (Mrays/s,
// Cash-Karp): 168 registers (three blocks) 14.4, 128: 15.5, 112: 15.4,
// 96: 15.3, 80: 14.7.
#ifndef OSIRIS_DF64_MAXREGS
#define OSIRIS_DF64_MAXREGS 128
#endif

struct KerrDF {
  using Ray = RayDF;
  static constexpr int kMaxRegs = OSIRIS_DF64_MAXREGS;
  static __device__ __forceinline__ Ray ray(const RayK& K) { return to_df(K); }
  static __device__ __forceinline__ void rhs(const Ray& K, df r, df th, df pr, df pth, df& dr,
                                             df& dth, df& dph, df& dpr, df& dpth,
                                             float& twoH) {
    rhs_df(K, r, th, pr, pth, dr, dth, dph, dpr, dpth, twoH);
  }
  static constexpr bool kTrackH = true;
  static constexpr bool kF32Stages = false;
  static constexpr double kLocateRel = 4e-16;
  static __device__ __forceinline__ float end_twoH(const Ray& K, const RayK&, const StateDF& y) {
    df dr, dth, dph, dpr, dpth;
    float twoH;
    rhs(K, y.r, y.th, y.pr, y.pth, dr, dth, dph, dpr, dpth, twoH);
    return twoH;
  }
};

struct QMetricDF {
  using Ray = RayQDF;
  static constexpr int kMaxRegs = OSIRIS_DF64_MAXREGS;
  static __device__ __forceinline__ Ray ray(const RayK& K) { return to_qdf(K); }
  static __device__ __forceinline__ void rhs(const Ray& K, df r, df th, df pr, df pth, df& dr,
                                             df& dth, df& dph, df& dpr, df& dpth,
                                             float& twoH) {
    rhs_q_df(K, r, th, pr, pth, dr, dth, dph, dpr, dpth, twoH);
  }
  static constexpr bool kTrackH = true;
  static constexpr bool kF32Stages = false;
  static constexpr double kLocateRel = 4e-16;
  static __device__ __forceinline__ float end_twoH(const Ray& K, const RayK&, const StateDF& y) {
    df dr, dth, dph, dpr, dpth;
    float twoH;
    rhs(K, y.r, y.th, y.pr, y.pth, dr, dth, dph, dpr, dpth, twoH);
    return twoH;
  }
};

template <class Met, int INTEG>
__global__ void __maxnreg__(Met::kMaxRegs) trace_df64_plain(const __grid_constant__ KernelArgs A) {
  trace_body_df<Met, false, INTEG>(A);
}

template <class Met, int INTEG>
__global__ void __maxnreg__(Met::kMaxRegs)
    trace_df64_persistent(const __grid_constant__ KernelArgs A) {
  trace_body_df<Met, true, INTEG>(A);
}

template <class Met, int INTEG>
static const void* df64_kernel(Kernel kind) {
  return kind == Kernel::kPersistent ? (const void*)trace_df64_persistent<Met, INTEG>
                                     : (const void*)trace_df64_plain<Met, INTEG>;
}

template <class Met>
static const void* df64_kernel(Kernel kind, int integrator) {
  return integrator == OSIRIS_RKDP45 ? df64_kernel<Met, OSIRIS_RKDP45>(kind)
                                     : df64_kernel<Met, OSIRIS_RKCK45>(kind);
}

static const void* select_df64(Kernel kind, int integrator, int spacetime) {
  return spacetime == OSIRIS_SPACETIME_QMETRIC ? df64_kernel<QMetricDF>(kind, integrator)
                                               : df64_kernel<KerrDF>(kind, integrator);
}

int launch_trace_df64(const KernelArgs& args, Kernel kind, int integrator, int grid, int block,
                      void* stream) {
  const int spacetime = args.reqs ? args.spacetime : args.single.spacetime;
  void* params[] = {const_cast<KernelArgs*>(&args)};
  return (int)cudaLaunchKernel(select_df64(kind, integrator, spacetime), dim3(grid),
                               dim3(block), params, 0, static_cast<cudaStream_t>(stream));
}

int occupancy_df64(Kernel kind, int integrator, int spacetime, int block, int* blocks_per_sm) {
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      blocks_per_sm, select_df64(kind, integrator, spacetime), block, 0);
}

}  // namespace osiris_impl
