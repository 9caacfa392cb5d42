"""Build the CUDA library in-tree: paper_2510_14712_gb300/_build/liblbm.so.

nvcc compiles each csrc/*.cu translation unit for sm_103a in parallel and
links them into one shared library exporting the C interface of
include/lbm.h.  Usage: ``python -m paper_2510_14712_gb300.build [--force]
[--bounds-check]``.  The bounds-check build (-DLBM_BOUNDS_CHECK, every
population access of the step kernels checked against its buffer) goes to
_build/liblbm_bc.so with its own objects.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "liblbm.so")
LIB_BC = os.path.join(OUT, "liblbm_bc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xptxas", "-O3"]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA 13 toolkit is required to build the library")
    return exe


def sources():
    return sorted(os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith(".cu"))


def extra_flags(src):
    """FP32-arithmetic kernel sets use the hardware reciprocal-based FP32
    division (about 2 ulp) instead of the IEEE-rounded one."""
    name = os.path.basename(src)
    if name.startswith("k_") and ("_fp32" in name or "_fp16" in name):
        return ["-prec-div=false"]
    return []


def _stale(srcs, lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = srcs + [os.path.join(SRC, f) for f in os.listdir(SRC)] + \
        [os.path.join(HERE, "..", "include", f) for f in ("lbm.h", "lbm_mlp.h")] + [os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force=False, verbose=False, bounds_check=False):
    srcs = sources()
    lib = LIB_BC if bounds_check else LIB
    if not force and not _stale(srcs, lib):
        return lib
    objdir = os.path.join(OUT, "bc") if bounds_check else OUT
    os.makedirs(objdir, exist_ok=True)
    cc = nvcc()
    defs = ["-DLBM_BOUNDS_CHECK"] if bounds_check else []

    def compile_one(src):
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        cmd = [cc] + ARCH + FLAGS + defs + extra_flags(src) + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + ".tmp"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, bounds_check="--bounds-check" in sys.argv))
