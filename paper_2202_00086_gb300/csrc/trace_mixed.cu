// Mixed-precision trace kernels. The six stage evaluations of Hamilton's
// equations run in FP32 (the GB300 FP32 pipe is ~70x the FP64 pipe); the
// state, the accumulation of each accepted increment, the error scale and
// the |H| constraint stay in FP64, and a step that starts near the horizon
// (r < 4) or at a polar turning point (|p_theta| < 1e-3) is taken entirely
// in FP64, where FP32 cancellation in N = Delta p_r^2 - P^2/Delta + ... is
// severe.
#include <cuda_runtime.h>

#include "trace_kernel.cuh"

namespace osiris_impl {

constexpr double kMixedFP64Radius = 4.0;
constexpr double kMixedFP64Ptheta = 1e-3;

struct RayK32 {
  float a, a2, aE, aL, E, L;
};

// The separated form of Hamilton's equations (see rhs64) in FP32.
__device__ __forceinline__ void rhs32(const RayK32& K, float r, float th, float pr, float pth,
                                      float& dr, float& dth, float& dph, float& dpr,
                                      float& dpth) {
  float s, c;
  sincosf(th, &s, &c);
  const float r2 = r * r;
  const float Delta = fmaf(r, r - 2.0f, K.a2);
  const float Sigma = fmaf(K.a2 * c, c, r2);
  const float P = fmaf(fmaf(r, r, K.a2), K.E, -K.aL);
  const float DS = Delta * Sigma;
  const float inv = __frcp_rn(DS * s);
  const float iSig = (Delta * s) * inv;
  const float iDel = (Sigma * s) * inv;
  const float is = DS * inv;
  const float W = fmaf(K.L, is, -K.aE * s);
  const float u = P * iDel;
  const float Dpr = Delta * pr;
  const float N = fmaf(Dpr, pr, fmaf(pth, pth, fmaf(W, W, -P * u)));
  const float NiS = N * iSig;
  dr = Dpr * iSig;
  dth = pth * iSig;
  dph = fmaf(W, is, K.a * u) * iSig;
  dpr = iSig * fmaf(1.0f - r, fmaf(u, u, pr * pr), fmaf(r, NiS, (r + r) * K.E * u));
  dpth = (c * iSig) * fmaf(W, fmaf(K.L, is * is, K.aE), -(K.a2 * s) * NiS);
}

struct StepperMixed {
  // FP32 stage values put ~1e-7 relative noise on a trial step's end point;
  // a bracket narrower than that cannot be resolved further
  static constexpr double kLocateRel = 2e-7;
  static constexpr bool kTrigTable = true;  // its FP64 steps use rhs64
  static constexpr bool kExpLogTable = false;
  struct RayCache {};
  struct LaneCache {};
  static __device__ __forceinline__ void prepare(const RayK&, RayCache&) {}
  static __device__ __forceinline__ void reset(LaneCache&) {}
  static __device__ __forceinline__ void accepted(LaneCache&) {}
  static __device__ __forceinline__ bool attempt(const RayK& K, const RayCache&, LaneCache&,
                                                 const State& y, double h,
                                                 State& o, State& d, double& twoH) {
    if (y.r < kMixedFP64Radius || fabs(y.pth) < kMixedFP64Ptheta) {
      ck_step64(K, y, h, o, d, twoH);
      return true;
    }
    using namespace ck;
    const RayK32 k{(float)K.a, (float)K.a2, (float)K.aE, (float)K.aL, (float)K.E, (float)K.L};
    const float hf = (float)h;
    const float yr = (float)y.r, yt = (float)y.th, ypr = (float)y.pr, ypt = (float)y.pth;
    float k1r, k1t, k1p, k1pr, k1pt;
    rhs32(k, yr, yt, ypr, ypt, k1r, k1t, k1p, k1pr, k1pt);
    float k2r, k2t, k2p, k2pr, k2pt;
    rhs32(k, fmaf(hf, (float)A21 * k1r, yr), fmaf(hf, (float)A21 * k1t, yt),
          fmaf(hf, (float)A21 * k1pr, ypr), fmaf(hf, (float)A21 * k1pt, ypt), k2r, k2t, k2p, k2pr,
          k2pt);
#define M3(c, y0) fmaf(hf, fmaf((float)A32, k2##c, (float)A31 * k1##c), y0)
    float k3r, k3t, k3p, k3pr, k3pt;
    rhs32(k, M3(r, yr), M3(t, yt), M3(pr, ypr), M3(pt, ypt), k3r, k3t, k3p, k3pr, k3pt);
#undef M3
#define M4(c, y0) fmaf(hf, fmaf((float)A43, k3##c, fmaf((float)A42, k2##c, (float)A41 * k1##c)), y0)
    float k4r, k4t, k4p, k4pr, k4pt;
    rhs32(k, M4(r, yr), M4(t, yt), M4(pr, ypr), M4(pt, ypt), k4r, k4t, k4p, k4pr, k4pt);
#undef M4
#define M5(c, y0)                                                                       \
  fmaf(hf, fmaf((float)A54, k4##c, fmaf((float)A53, k3##c, fmaf((float)A52, k2##c,     \
                                                                 (float)A51 * k1##c))), \
       y0)
    float k5r, k5t, k5p, k5pr, k5pt;
    rhs32(k, M5(r, yr), M5(t, yt), M5(pr, ypr), M5(pt, ypt), k5r, k5t, k5p, k5pr, k5pt);
#undef M5
#define M6(c, y0)                                                                            \
  fmaf(hf,                                                                                   \
       fmaf((float)A65, k5##c,                                                               \
            fmaf((float)A64, k4##c,                                                          \
                 fmaf((float)A63, k3##c, fmaf((float)A62, k2##c, (float)A61 * k1##c)))), \
       y0)
    float k6r, k6t, k6p, k6pr, k6pt;
    rhs32(k, M6(r, yr), M6(t, yt), M6(pr, ypr), M6(pt, ypt), k6r, k6t, k6p, k6pr, k6pt);
#undef M6
#define INC(c) (hf * fmaf((float)B6, k6##c, fmaf((float)B4, k4##c, fmaf((float)B3, k3##c, (float)B1 * k1##c))))
#define DLT(c)                                                                              \
  (hf * fmaf((float)D6, k6##c,                                                              \
             fmaf((float)D5, k5##c,                                                         \
                  fmaf((float)D4, k4##c, fmaf((float)D3, k3##c, (float)D1 * k1##c)))))
    o.r = y.r + (double)INC(r);
    o.th = y.th + (double)INC(t);
    o.ph = y.ph + (double)INC(p);
    o.pr = y.pr + (double)INC(pr);
    o.pth = y.pth + (double)INC(pt);
    d.r = (double)DLT(r);
    d.th = (double)DLT(t);
    d.ph = (double)DLT(p);
    d.pr = (double)DLT(pr);
    d.pth = (double)DLT(pt);
#undef INC
#undef DLT
    twoH = twoH_kerr_direct(K, y);
    return false;
  }
  static __device__ __forceinline__ double twoH(const RayK& K, const State& y) {
    return twoH_kerr_direct(K, y);
  }
};

constexpr int kMaxBlock = 256;

__global__ void __launch_bounds__(kMaxBlock) trace_mixed_plain(const __grid_constant__ KernelArgs A) {
  trace_body<StepperMixed, false>(A);
}

__global__ void __launch_bounds__(kMaxBlock) trace_mixed_persistent(const __grid_constant__ KernelArgs A) {
  trace_body<StepperMixed, true>(A);
}

int launch_trace_mixed(const KernelArgs& args, Kernel kind, int, int grid, int block,
                       void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (kind == Kernel::kPersistent)
    trace_mixed_persistent<<<grid, block, 0, s>>>(args);
  else
    trace_mixed_plain<<<grid, block, 0, s>>>(args);
  return (int)cudaGetLastError();
}

int occupancy_mixed(Kernel kind, int, int, int block, int* blocks_per_sm) {
  const void* fn = (kind == Kernel::kPersistent) ? (const void*)trace_mixed_persistent
                                                 : (const void*)trace_mixed_plain;
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block, 0);
}

}  // namespace osiris_impl
