"""Build the sm_103a shared library libfirert.so in-tree with nvcc.

The library is the product's C ABI (include/firert.h); the Python binding
loads it with ctypes. Only nvcc and the CUDA runtime are needed. With
debug=True the same sources build libfirert_debug.so with FIRERT_DEBUG: the
fit kernels check their indices and shared-memory regions and report a
failed check as FIRE_ERR_BOUNDS instead of making the access.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = [os.path.join(HERE, "csrc", f) for f in ("api.cu", "kernels_lm.cu", "kernels_aux.cu",
                                               "kernels_gemm.cu", "kernels_mlp.cu", "mlp.cu", "batch.cu",
                                         "noalloc.cu", "alloc.cu", "peaks.cu")]
DEPS = SRC + [os.path.join(HERE, "csrc", f) for f in ("internal.cuh", "model.cuh", "mlp_internal.h", "tc.cuh",
                                                       "ctx_internal.h")] + \
    [os.path.join(ROOT, "include", "firert.h")]
LIB = os.path.join(HERE, "libfirert.so")
LIB_DEBUG = os.path.join(HERE, "libfirert_debug.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "-Xcompiler", "-fPIC", "-shared", "--expt-relaxed-constexpr"]


def build(force=False, verbose=False, debug=False):
    lib = LIB_DEBUG if debug else LIB
    if not force and os.path.exists(lib):
        t = os.path.getmtime(lib)
        if all(os.path.getmtime(d) <= t for d in DEPS):
            return lib
    objs = []
    for s in SRC:
        o = os.path.join(HERE, "_build_debug" if debug else "_build", os.path.basename(s) + ".o")
        os.makedirs(os.path.dirname(o), exist_ok=True)
        cmd = [NVCC] + [f for f in FLAGS if f != "-shared"] + (["-DFIRERT_DEBUG"] if debug else []) + \
            ["-c", s, "-o", o]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        subprocess.check_call(cmd)
        objs.append(o)
    subprocess.check_call([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-shared",
                           "-Xcompiler", "-fPIC", "-o", lib] + objs)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
