"""Build libchfpe.so in-tree for sm_103a with nvcc (no JIT, no torch extension machinery)."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libchfpe.so")
SOURCES = [os.path.join(HERE, "csrc", f) for f in ("chfpe.cu", "noalloc.cu", "surrogate.cu")]
DEPS = SOURCES + [os.path.join(HERE, "csrc", f) for f in ("kernels.cuh", "bulk.cuh", "persistent.cuh")] + [os.path.join(ROOT, "include", "chfpe.h")]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def flags(verbose: bool = False):
    f = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "-Xcompiler", "-fPIC", "-shared", "--expt-relaxed-constexpr", "-lcudart"]
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in DEPS)


def build(force: bool = False, verbose: bool = False) -> str:
    if force or stale():
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [NVCC] + flags(verbose) + SOURCES + ["-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose="-v" in sys.argv)
    print(LIB)
