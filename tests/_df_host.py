"""Host builds of device code for CPU tests: the double-float (df64) headers
and the FP64 evaluation header (trace_device.cuh). The FP32 intrinsics are
mapped to plain IEEE single operations (the host compiler is told not to
contract a*b+c, so every operation rounds once, as the intrinsics do on the
GPU); for trace_device.cuh, a block of one thread stands in for the CUDA
built-ins (shared tables become function-local statics, filled by that one
thread)."""
import pathlib
import shutil
import subprocess

import pytest

ROOT = pathlib.Path(__file__).resolve().parent.parent
CSRC = ROOT / "paper_2202_00086_gb300" / "csrc"

SHIMS = r"""
#include <math.h>
#include <cstdint>
#include <cstring>
#include <cstdio>
#define __device__
#define __forceinline__ inline
static inline float __fadd_rn(float a, float b) { return a + b; }
static inline float __fsub_rn(float a, float b) { return a - b; }
static inline float __fmul_rn(float a, float b) { return a * b; }
static inline float __fdividef(float a, float b) { return a / b; }
static inline float osiris_host_expf(float x) { return expf(x); }
static inline float osiris_host_logf(float x) { return logf(x); }
#define __expf osiris_host_expf
#define __logf osiris_host_logf
static inline float __double2float_rn(double x) { return (float)x; }
static inline unsigned __float_as_uint(float x) { unsigned u; std::memcpy(&u, &x, 4); return u; }
static inline float __uint_as_float(unsigned u) { float x; std::memcpy(&x, &u, 4); return x; }
static inline float __int_as_float(int i) { float x; std::memcpy(&x, &i, 4); return x; }
"""


DEVICE_SHIMS = r"""
#include <cmath>
#define __shared__ static
#define __host__
struct osiris_dim3 { unsigned x, y, z; };
static const osiris_dim3 threadIdx = {0, 0, 0};
static const osiris_dim3 blockDim = {1, 1, 1};
static inline void __syncthreads() {}
struct double2 { double x, y; };
static inline double2 make_double2(double x, double y) { double2 r; r.x = x; r.y = y; return r; }
struct float4 { float x, y, z, w; };
static inline float4 make_float4(float x, float y, float z, float w) {
  float4 r; r.x = x; r.y = y; r.z = z; r.w = w; return r;
}
static inline int __clzll(long long v) { return v == 0 ? 64 : __builtin_clzll((unsigned long long)v); }
static inline long long __double_as_longlong(double x) {
  long long b; std::memcpy(&b, &x, 8); return b;
}
static inline double __longlong_as_double(long long b) {
  double x; std::memcpy(&x, &b, 8); return x;
}
static inline int __double2hiint(double x) { return (int)(__double_as_longlong(x) >> 32); }
static inline int __float_as_int(float x) { int i; std::memcpy(&i, &x, 4); return i; }
static inline double __drcp_rn(double x) { return 1.0 / x; }
template <class T> static inline T __ldg(const T* p) { return *p; }
template <class T> static inline T __shfl_xor_sync(unsigned, T v, int) { return v; }
static inline unsigned long long atomicAdd(unsigned long long* p, unsigned long long v) {
  const unsigned long long o = *p; *p += v; return o;
}
static inline unsigned long long atomicMax(unsigned long long* p, unsigned long long v) {
  const unsigned long long o = *p; if (v > o) *p = v; return o;
}
"""


def build(tmp_path_factory, name, source, device_shims=False):
    """Compile SHIMS (+ DEVICE_SHIMS) + source (which includes headers from
    csrc/) to an executable; skips the test when no host C++ compiler is
    present."""
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp(name)
    (d / "h.cpp").write_text(SHIMS + (DEVICE_SHIMS if device_shims else "") + source)
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I" + str(CSRC),
                    "-I" + str(ROOT / "include"), str(d / "h.cpp"), "-o", str(d / "h")],
                   check=True)
    return d / "h"
