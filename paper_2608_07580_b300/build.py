"""Build the sm_103a shared library libfirert.so in-tree with nvcc.

The library is the product's C ABI (include/firert.h); the Python binding
loads it with ctypes. Only nvcc and the CUDA runtime are needed.
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
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "-Xcompiler", "-fPIC", "-shared", "--expt-relaxed-constexpr"]


def build(force=False, verbose=False):
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in DEPS):
            return LIB
    objs = []
    for s in SRC:
        o = os.path.join(HERE, "_build", os.path.basename(s) + ".o")
        os.makedirs(os.path.dirname(o), exist_ok=True)
        cmd = [NVCC] + [f for f in FLAGS if f != "-shared"] + ["-dc" if False else "-c", s, "-o", o]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        subprocess.check_call(cmd)
        objs.append(o)
    subprocess.check_call([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-shared",
                           "-Xcompiler", "-fPIC", "-o", LIB] + objs)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
