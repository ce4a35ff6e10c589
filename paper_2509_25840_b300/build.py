"""Build libchfpe.so in-tree for sm_103a with nvcc (no JIT, no torch extension machinery): every
translation unit is compiled to an object in parallel, then the objects are linked."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libchfpe.so")
CSRC = os.path.join(HERE, "csrc")
SOURCES = [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith(".cu")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")] + \
    [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def flags(verbose: bool = False):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]
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
        tag = f".tmp{os.getpid()}"
        objs = [os.path.join(CSRC, os.path.basename(s)[:-3] + tag + ".o") for s in SOURCES]
        procs = [subprocess.Popen([NVCC] + flags(verbose) + ["-c", s, "-o", o])
                 for s, o in zip(SOURCES, objs)]
        rcs = [p.wait() for p in procs]
        try:
            if any(rcs):
                raise subprocess.CalledProcessError(max(rcs), "nvcc -c")
            tmp = LIB + tag
            subprocess.run([NVCC] + ARCH + ["-shared", "-Xcompiler", "-fPIC"] + objs +
                           ["-lcudart", "-o", tmp], check=True)
            os.replace(tmp, LIB)
        finally:
            for o in objs:
                if os.path.exists(o):
                    os.remove(o)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose="-v" in sys.argv)
    print(LIB)
