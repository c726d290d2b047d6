"""Build the CUDA library libsmcrt for sm_103a (in-tree, no cmake).

Translation units and their floating-point flags:
  smcrt_k64.cu   FP64 packet kernel, -fmad=false (no FMA contraction, so the
                 kernel's arithmetic is the reference's IEEE sequence);
  smcrt_k32.cu   mixed kernel, approximate FP32 division/sqrt, FTZ; the
                 multiply-adds are fused where the source writes them
                 (__fmaf_rn in the distances, moves, tally set-up and
                 scattering: 3 % on the layered slab) or the front end
                 contracts them, and nowhere else: the assembler
                 may not fuse plain multiply / add pairs (--fmad=false),
                 because it fused them differently under different register
                 budgets, and every instantiation must give the same bits;
  smcrt_util.cu  helper kernels;
  smcrt_api.cpp  host runtime (C-ABI), -ffp-contract=off.
"""
from __future__ import annotations

import os
import platform
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(BUILD, f"libsmcrt_{platform.machine()}.so")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
          f"-I{os.path.join(ROOT, 'include')}"]

UNITS = {
    "smcrt_k64.cu": ["-fmad=false"],
    "smcrt_k32.cu": ["-ftz=true", "-prec-div=false", "-prec-sqrt=false", "-Xptxas", "--fmad=false"],
    "smcrt_util.cu": [],
    "smcrt_noalloc.cu": [],
    "smcrt_microbench.cu": [],
}
HEADERS = ["smcrt_internal.h", "smcrt_kernel.cuh"]


def _newer(src_list, target):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in src_list)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "smcrt.h")]
    objs, jobs = [], []
    arch = platform.machine()
    for unit, flags in UNITS.items():
        src = os.path.join(CSRC, unit)
        obj = os.path.join(BUILD, f"{unit}.{arch}.o")
        objs.append(obj)
        if force or _newer([src] + hdrs, obj):
            extra = ["-Xptxas", "-v"] if verbose else []
            jobs.append([NVCC] + ARCH + COMMON + flags + extra + ["-c", src, "-o", obj])
    api_src = os.path.join(CSRC, "smcrt_api.cpp")
    api_obj = os.path.join(BUILD, f"smcrt_api.{arch}.o")
    objs.append(api_obj)
    if force or _newer([api_src] + hdrs, api_obj):
        jobs.append(["g++", "-std=c++17", "-O2", "-fPIC", "-ffp-contract=off", "-Wall",
                     f"-I{os.path.join(CUDA, 'include')}", f"-I{os.path.join(ROOT, 'include')}",
                     "-c", api_src, "-o", api_obj])
    if jobs:
        with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            outs = list(ex.map(_run, jobs))
        if verbose:
            for o in outs:
                sys.stdout.write(o)
    if force or _newer(objs, LIB):
        tmp = LIB + f".tmp{os.getpid()}"
        _run([NVCC] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs +
             ["-Xlinker", f"-rpath,{os.path.join(CUDA, 'lib64')}", "-lpthread"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
