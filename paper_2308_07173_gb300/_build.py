"""Compile libpc.so in-tree for sm_103a with nvcc (no torch extension).

Translation units compile in parallel, then link into
``paper_2308_07173_gb300/libpc.so`` with the CUDA runtime linked statically,
so the library loads on any machine with the NVIDIA driver (and, without a
GPU, still loads for symbol checks).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libpc.so")

SOURCES = ["knn_cov.cu", "knn_window.cu", "knn_union.cu", "knn_union_win.cu", "pc_api.cu", "grid_build.cu",
           "noalloc.cu", "gicp.cu", "wall.cu", "delta.cu"]
HEADERS = ["pc_device.cuh", "pc_internal.h", "pc_search.cuh", "knn_kernels.cuh"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# --fmad=false: no implicit contraction anywhere, so every fused multiply-add
# in the kernels is an explicit __fmaf_rn and results are reproducible across
# inlining contexts.  IEEE division/sqrt and no flush-to-zero (nvcc defaults
# without --use_fast_math) are spelled out.
NVFLAGS = ARCH + [
    "-O3",
    "-lineinfo",
    "-std=c++17",
    "--fmad=false",
    "-ftz=false",
    "-prec-div=true",
    "-prec-sqrt=true",
    "-Xcompiler",
    "-fPIC,-fvisibility=hidden,-O2",
    "-I",
    INCLUDE,
    "-I",
    CSRC,
]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpc.so")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "pc.h"), __file__]
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            jobs.append([cc, *NVFLAGS, *extra, "-c", s, "-o", o])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            futs = [ex.submit(subprocess.run, j, capture_output=True, text=True) for j in jobs]
            for j, f in zip(jobs, futs):
                r = f.result()
                if verbose or r.returncode != 0:
                    sys.stderr.write(r.stdout + r.stderr)
                if r.returncode != 0:
                    raise RuntimeError(f"nvcc failed: {' '.join(j)}")
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fPIC"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link of libpc.so failed")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
