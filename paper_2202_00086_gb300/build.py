"""Build the CUDA library libosiris.so (sm_103a) in-tree, and its
bounds-checked twin libosiris_checked.so (the same sources with
-DOSIRIS_CHECKED: every ray's queue, request and pixel indices are checked
before use and failures are counted in the stats array instead of trapping).

Each translation unit is compiled by nvcc in parallel, then linked into
paper_2202_00086_gb300/_build/libosiris.so (_build/checked/ for the checked
twin). ptxas resource usage (registers, spills, stack) is written to
_build/ptxas.txt.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libosiris.so")
OUT_CHECKED = os.path.join(OUT, "checked")
LIB_CHECKED = os.path.join(OUT, "libosiris_checked.so")
SOURCES = ["osiris_api.cu", "trace_fp64.cu", "trace_mixed.cu", "trace_df64.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
         "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]

# The FP64 and mixed units write every fused multiply-add explicitly; with
# contraction off the compiler cannot fuse a product into a sum differently in
# different kernels, so every kernel computes bit-identical results.
TU_FLAGS = {"trace_fp64.cu": ["-fmad=false"], "trace_mixed.cu": ["-fmad=false"]}


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _newest_input():
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    paths.append(os.path.join(ROOT, "include", "osiris.h"))
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


def _variant(checked):
    return ((OUT_CHECKED, LIB_CHECKED, ["-DOSIRIS_CHECKED"]) if checked else (OUT, LIB, []))


def _stale(lib):
    return not os.path.exists(lib) or os.path.getmtime(lib) < _newest_input()


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile libosiris.so (or, with checked, libosiris_checked.so) if it is
    missing or stale; return its path."""
    return build_all(force=force, verbose=verbose, variants=(checked,))[0]


def build_all(force: bool = False, verbose: bool = False, variants=(False, True)):
    """Compile the requested library variants (False: libosiris.so, True:
    the bounds-checked twin), every translation unit of all of them in one
    parallel pool; return their paths."""
    todo = [c for c in variants if force or _stale(_variant(c)[1])]
    if not todo:
        return [_variant(c)[1] for c in variants]
    nvcc = _nvcc()
    jobs = []
    for c in todo:
        out, _, extra = _variant(c)
        os.makedirs(out, exist_ok=True)
        jobs += [(c, src, out, extra) for src in SOURCES]

    def compile_one(job):
        c, src, out, extra = job
        obj = os.path.join(out, src.replace(".cu", ".o"))
        cmd = ([nvcc] + ARCH + FLAGS + extra + TU_FLAGS.get(src, []) +
               ["-c", os.path.join(CSRC, src), "-o", obj])
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, p.stdout, p.stderr))
        return obj, p.stderr

    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        results = list(ex.map(compile_one, jobs))
    for c in todo:
        out, lib, _ = _variant(c)
        mine = [(r, j) for r, j in zip(results, jobs) if j[0] == c]
        with open(os.path.join(out, "ptxas.txt"), "w") as f:
            for (obj, log), job in mine:
                f.write("== %s\n%s\n" % (job[1], log))
        tmp = lib + ".tmp%d" % os.getpid()
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + [obj for (obj, _), _ in mine]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("link failed:\n%s%s" % (p.stdout, p.stderr))
        os.replace(tmp, lib)
    if verbose:
        print(open(os.path.join(OUT, "ptxas.txt")).read())
    return [_variant(c)[1] for c in variants]


if __name__ == "__main__":
    print(build_all(force="--force" in sys.argv, verbose="-v" in sys.argv))
