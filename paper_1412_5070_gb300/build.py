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
# (source, extra nvcc flags): the thin contraction instances are one source
# compiled in seven parts, so that they build in parallel
SOURCES = [(os.path.join(CSRC, "f12int.cu"), ())] + \
    [(os.path.join(CSRC, "thin_inst.cu"), ("-DF12_THIN_PART=%d" % p,)) for p in range(7)] + \
    [(os.path.join(CSRC, "peak.cu"), ()), (os.path.join(CSRC, "termlist.cpp"), ())]
DEPS = sorted({src for src, _ in SOURCES}) + [os.path.join(CSRC, f) for f in (
    "aux.cuh", "auxtab.h", "engine.cuh", "termlist.h", "kernel_common.cuh", "thin.cuh")] + \
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
    """Compile every source to an object in parallel (one nvcc process each),
    then link the shared library."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = nvcc_path()
    tag = ".tmp%d" % os.getpid()
    objs, procs = [], []
    for k, (src, flags) in enumerate(SOURCES):
        obj = os.path.join(BUILD, "%s.%d%s.o" % (os.path.basename(src), k, tag))
        cmd = [nvcc, "-O3", "-lineinfo", "-std=c++17", *ARCH, "-Xcompiler", "-fPIC", *flags, "-c", "-o", obj, src,
               *extra]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        objs.append(obj)
        procs.append((cmd, subprocess.Popen(cmd)))
    failed = [cmd for cmd, p in procs if p.wait() != 0]
    if failed:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
        raise subprocess.CalledProcessError(1, failed[0])
    tmp = LIB + tag
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    try:
        subprocess.run(cmd, check=True)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=("-Xptxas", "-v") if "--ptxas" in sys.argv else ()))
