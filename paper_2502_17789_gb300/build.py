"""Build libidg.so (the CUDA library behind include/idg.h) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel into _build/, then
linked into paper_2502_17789_gb300/libidg.so.  Host code is compiled without
floating-point contraction so the planner rounds identically on x86 and Arm.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libidg.so")
SOURCES = (["planner.cpp", "gridder.cu", "fft.cu", "degridder.cu", "idg_api.cu", "noalloc.cu", "image.cu", "probe.cu"]
           + [f"gridder_l{L}.cu" for L in (32, 64, 96, 128)] + [f"degridder_l{L}.cu" for L in (32, 64, 96, 128)]
           + [f"degridder_tc_l{L}.cu" for L in (32, 64, 96, 128)]
           + [f"gridder_tc_l{L}.cu" for L in (32, 64, 96, 128)])
HEADERS = ["idg_internal.h", "kernels_common.cuh", "gridder_kernels.cuh", "degridder_kernels.cuh",
           "degridder_tc_kernels.cuh", "gridder_tc_kernels.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc")
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off,-fno-fast-math",
                "-I", os.path.join(ROOT, "include")]


def _newest_input() -> float:
    paths = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "idg.h"), __file__]
    return max(os.path.getmtime(p) for p in paths)


def _compile(src: str, verbose: bool) -> str:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [NVCC] + FLAGS + (["-Xptxas", "-v"] if verbose and src.endswith(".cu") else []) + \
        ["-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose:
        print(r.stderr)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    tmp = LIB + ".tmp"
    # cuFFT (the master-grid transform of the image-domain wrapper), found at run time next to the toolkit
    import shutil
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(shutil.which(NVCC) or NVCC))), "lib64")
    r = subprocess.run([NVCC] + ARCH + ["-shared", "-o", tmp] + objs +
                       ["-L" + cuda_lib, "-lcufft", "-Xlinker", "-rpath," + cuda_lib],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
