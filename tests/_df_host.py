"""Host builds of the double-float (df64) device code for CPU tests: the FP32
intrinsics it uses are mapped to plain IEEE single operations (the host
compiler is told not to contract a*b+c, so every operation rounds once, as
the intrinsics do on the GPU)."""
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
static inline float __double2float_rn(double x) { return (float)x; }
static inline unsigned __float_as_uint(float x) { unsigned u; std::memcpy(&u, &x, 4); return u; }
static inline float __uint_as_float(unsigned u) { float x; std::memcpy(&x, &u, 4); return x; }
static inline float __int_as_float(int i) { float x; std::memcpy(&x, &i, 4); return x; }
"""


def build(tmp_path_factory, name, source):
    """Compile SHIMS + source (which includes headers from csrc/) to an
    executable; skips the test when no host C++ compiler is present."""
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp(name)
    (d / "h.cpp").write_text(SHIMS + source)
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I" + str(CSRC),
                    "-I" + str(ROOT / "include"), str(d / "h.cpp"), "-o", str(d / "h")],
                   check=True)
    return d / "h"
