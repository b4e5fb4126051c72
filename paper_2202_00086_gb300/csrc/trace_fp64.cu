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

// Roofline probes: kProbeChains independent chains of one arithmetic
// operation per thread (OP 0: fused multiply-add a = a b + c, 1: multiply
// a = a b, 2: add a = a + c, 3: the multiply issued as a fused multiply-add
// with a zero addend, 4: the add issued as a fused multiply-add by one), the
// chain step unrolled so that each loop trip
// issues 4 kProbeChains operations back to back. The operands b and c are
// per-thread values, so the compiler cannot hoist or fold them. This
// translation unit is compiled with contraction off, so a multiply or an add
// stays one instruction of the pipe under test.
constexpr int kProbeChains = 16;
constexpr int kProbeBlock = 256;

template <typename T, int OP>
__device__ __forceinline__ T probe_op(T a, T b, T c) {
  if (OP == 0) return fma(a, b, c);
  if (OP == 1) return a * b;
  if (OP == 2) return a + c;
  if (OP == 3) return mul_as_fma(a, b);
  return add_as_fma(a, c);
}

template <typename T, int OP>
__global__ void __launch_bounds__(kProbeBlock) pipe_probe_kernel(double* out, T b0, T c0,
                                                                 int iters) {
  const T t = (T)threadIdx.x * (T)1e-6;
  const T b = b0 + t * (T)1e-3, c = c0 + t;
  T a[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) a[k] = t + (T)k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int k = 0; k < kProbeChains; ++k) a[k] = probe_op<T, OP>(a[k], b, c);
  }
  T sum = (T)0;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) sum += a[k];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = (double)sum;
}

template <typename T, int OP>
static int launch_probe_t(int64_t n_threads, int iters, double* out, cudaStream_t s) {
  const int grid = (int)(n_threads / kProbeBlock);
  const T b = (T)0.999999, c = (T)1e-7;
  pipe_probe_kernel<T, OP><<<grid, kProbeBlock, 0, s>>>(out, b, c, iters);
  return (int)cudaGetLastError();
}

template <typename T>
static const void* probe_kernel_t(int op) {
  switch (op) {
    case 0: return (const void*)pipe_probe_kernel<T, 0>;
    case 1: return (const void*)pipe_probe_kernel<T, 1>;
    case 2: return (const void*)pipe_probe_kernel<T, 2>;
    case 3: return (const void*)pipe_probe_kernel<T, 3>;
    default: return (const void*)pipe_probe_kernel<T, 4>;
  }
}

template <typename T>
static int launch_probe_op(int op, int64_t n_threads, int iters, double* out, cudaStream_t s) {
  switch (op) {
    case 0: return launch_probe_t<T, 0>(n_threads, iters, out, s);
    case 1: return launch_probe_t<T, 1>(n_threads, iters, out, s);
    case 2: return launch_probe_t<T, 2>(n_threads, iters, out, s);
    case 3: return launch_probe_t<T, 3>(n_threads, iters, out, s);
    default: return launch_probe_t<T, 4>(n_threads, iters, out, s);
  }
}

int launch_pipe_probe(int precision, int op, int64_t n_threads, int iters, double* out,
                      void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return precision == OSIRIS_FP64 ? launch_probe_op<double>(op, n_threads, iters, out, s)
                                  : launch_probe_op<float>(op, n_threads, iters, out, s);
}

int probe_resident_blocks(int precision, int op, int* blocks_per_sm) {
  const void* fn = precision == OSIRIS_FP64 ? probe_kernel_t<double>(op)
                                            : probe_kernel_t<float>(op);
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, kProbeBlock, 0);
}

}  // namespace osiris_impl
