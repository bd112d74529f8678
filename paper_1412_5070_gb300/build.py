"""Build the CUDA library in-tree: paper_1412_5070_gb300/_build/libf12int.so.

One nvcc invocation, one -gencode (sm_103a), no CMake.  Run on each machine
that loads the library (the GPU machine builds its own copy).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libf12int.so")
SOURCES = [os.path.join(CSRC, "f12int.cu"), os.path.join(CSRC, "peak.cu"), os.path.join(CSRC, "termlist.cpp")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in ("aux.cuh", "auxtab.h", "engine.cuh", "termlist.h")] + \
    [os.path.join(os.path.dirname(HERE), "include", "f12int.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in DEPS if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc_path(), "-O3", "-lineinfo", "-std=c++17", *ARCH, "-Xcompiler", "-fPIC", "-shared",
           "-o", tmp, *SOURCES, "-lcudart", *extra]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=("-Xptxas", "-v") if "--ptxas" in sys.argv else ()))
