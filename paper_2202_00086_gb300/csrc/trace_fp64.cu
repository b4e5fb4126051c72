// FP64 trace kernels: every operation of the integrator in double precision.
#include <cuda_runtime.h>

#include "trace_kernel.cuh"

namespace osiris_impl {

template <int INTEG, class Met>
struct StepperFP64;

// Cash-Karp: every attempt evaluates its six stages.
template <class Met>
struct StepperFP64<OSIRIS_RKCK45, Met> {
  static constexpr double kLocateRel = 0.0;
  static constexpr bool kTrigTable = Met::kTrigTable;
  static constexpr bool kExpLogTable = Met::kExpLogTable;
  struct RayCache {};
  struct LaneCache {};
  static __device__ __forceinline__ void prepare(const RayK&, RayCache&) {}
  static __device__ __forceinline__ void reset(LaneCache&) {}
  static __device__ __forceinline__ void accepted(LaneCache&) {}
  static __device__ __forceinline__ bool attempt(const RayK& K, const RayCache&, LaneCache&,
                                                 const State& y, double h, State& o, State& d,
                                                 double& twoH) {
    ck_step64<Met>(K, y, h, o, d, twoH);
    return true;
  }
  static __device__ __forceinline__ double twoH(const RayK& K, const State& y) {
    return twoH64<Met>(K, y);
  }
};

// Dormand-Prince: k1 is carried from the previous accepted attempt's seventh
// stage; it is evaluated only when a ray starts or resumes (a warp evaluates
// it when any of its lanes needs it).
template <class Met>
struct StepperFP64<OSIRIS_RKDP45, Met> {
  static constexpr double kLocateRel = 0.0;
  static constexpr bool kTrigTable = Met::kTrigTable;
  static constexpr bool kExpLogTable = Met::kExpLogTable;
  struct RayCache {};
  struct LaneCache {
    Deriv k1, k7;
    bool valid;
  };
  static __device__ __forceinline__ void prepare(const RayK&, RayCache&) {}
  static __device__ __forceinline__ void reset(LaneCache& c) { c.valid = false; }
  static __device__ __forceinline__ void accepted(LaneCache& c) { c.k1 = c.k7; }
  static __device__ __forceinline__ bool attempt(const RayK& K, const RayCache&, LaneCache& c,
                                                 const State& y, double h, State& o, State& d,
                                                 double& twoH) {
    if (!c.valid) {
      rhs64_at<Met>(K, y, c.k1);
      c.valid = true;
    }
    twoH = c.k1.twoH;
    dp_step64<Met>(K, y, h, c.k1, o, d, c.k7);
    return true;
  }
  static __device__ __forceinline__ double twoH(const RayK& K, const State& y) {
    return twoH64<Met>(K, y);
  }
};


template <int INTEG, class Met>
__global__ void __maxnreg__(Met::kMaxRegs) trace_fp64_plain(const __grid_constant__ KernelArgs A) {
  trace_body<StepperFP64<INTEG, Met>, false>(A);
}

template <int INTEG, class Met>
__global__ void __maxnreg__(Met::kMaxRegs) trace_fp64_persistent(const __grid_constant__ KernelArgs A) {
  trace_body<StepperFP64<INTEG, Met>, true>(A);
}

template <int INTEG, class Met>
static const void* fp64_kernel(Kernel kind) {
  return kind == Kernel::kPersistent ? (const void*)trace_fp64_persistent<INTEG, Met>
                                     : (const void*)trace_fp64_plain<INTEG, Met>;
}

static const void* select_fp64(Kernel kind, int integrator, int spacetime) {
  if (spacetime == OSIRIS_SPACETIME_QMETRIC)
    return integrator == OSIRIS_RKDP45 ? fp64_kernel<OSIRIS_RKDP45, QMetric>(kind)
                                       : fp64_kernel<OSIRIS_RKCK45, QMetric>(kind);
  return integrator == OSIRIS_RKDP45 ? fp64_kernel<OSIRIS_RKDP45, KerrMetric>(kind)
                                     : fp64_kernel<OSIRIS_RKCK45, KerrMetric>(kind);
}

int launch_trace_fp64(const KernelArgs& args, Kernel kind, int integrator, int grid, int block,
                      void* stream) {
  const int spacetime = args.reqs ? args.spacetime : args.single.spacetime;
  const void* fn = select_fp64(kind, integrator, spacetime);
  void* params[] = {const_cast<KernelArgs*>(&args)};
  return (int)cudaLaunchKernel(fn, dim3(grid), dim3(block), params, 0,
                               static_cast<cudaStream_t>(stream));
}

int occupancy_fp64(Kernel kind, int integrator, int spacetime, int block, int* blocks_per_sm) {
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      blocks_per_sm, select_fp64(kind, integrator, spacetime), block, 0);
}

// Roofline probe: 8 independent FMA chains per thread.
template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(double* out, T b, T c, int iters) {
  T a0 = (T)threadIdx.x * (T)1e-3, a1 = a0 + (T)1, a2 = a0 + (T)2, a3 = a0 + (T)3;
  T a4 = a0 + (T)4, a5 = a0 + (T)5, a6 = a0 + (T)6, a7 = a0 + (T)7;
  for (int i = 0; i < iters; ++i) {
    a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
    a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
  }
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = (double)(a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7);
}

int launch_fma_probe(int precision, int64_t n_threads, int iters, double* out, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int grid = (int)(n_threads / 256);
  if (precision == OSIRIS_FP64)
    fma_probe_kernel<double><<<grid, 256, 0, s>>>(out, 0.999999, 1e-7, iters);
  else
    fma_probe_kernel<float><<<grid, 256, 0, s>>>(out, 0.999999f, 1e-7f, iters);
  return (int)cudaGetLastError();
}

}  // namespace osiris_impl
