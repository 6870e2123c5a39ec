"""Builds libmg.so in place (nvcc, sm_103a).  Run: python -m paper_2608_29082_b300.build"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libmg.so")
LIB_DEBUG = os.path.join(HERE, "libmg_debug.so")  # -DMG_BOUNDS_CHECK

SOURCES = ["mg_api.cu", "setup_host.cpp", "noalloc.cu", "features2.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def sources() -> list[str]:
    return [os.path.join(CSRC, s) for s in SOURCES]


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    deps = sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(INCLUDE, "mg.h"))
    return all(os.path.getmtime(d) <= t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False,
          debug: bool = False) -> str:
    """libmg.so, or with debug=True libmg_debug.so: the same sources with
    every table-driven gather index checked (-DMG_BOUNDS_CHECK)."""
    lib = LIB_DEBUG if debug else LIB
    if not force and up_to_date(lib):
        return lib
    # -fmad=false: the kernels fuse multiply-adds only where they call fma()
    # explicitly, so every launch form of a step rounds identically
    cmd = [nvcc(), "-O3", "-std=c++17", *ARCH, "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC,-O2",
           "-shared", "-I", INCLUDE, "-I", CSRC, "-o", lib + ".tmp", *sources(), "-lcudart", "-ldl"]
    if debug:
        cmd.insert(1, "-DMG_BOUNDS_CHECK")
    if ptxas_v:
        cmd.insert(1, "-Xptxas=-v")
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed ({r.returncode}):\n{r.stdout}\n{r.stderr}")
    if ptxas_v or verbose:
        print(r.stderr, file=sys.stderr)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_v="--ptxas-v" in sys.argv,
                debug="--debug" in sys.argv))
