"""Build libpcg.so in-tree for sm_103a (B300).

The CUDA sources are compiled with nvcc for ``compute_103a``/``sm_103a`` only;
the host-side factor build is compiled by g++ without floating-point
contraction so that its arithmetic is plain IEEE binary64.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libpcg.so")
ROOT = os.path.dirname(HERE)
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["api.cu", "solve.cu", "shard.cu", "server.cu", "noalloc.cu", "measure.cu", "kernels_f64_64.cu", "kernels_f64_128.cu",
              "kernels_f32_64.cu", "kernels_f32_128.cu", "kernels_exact.cu", "kernels_f64_wide.cu"]
CPP_SOURCES = ["ainv_host.cpp"]
HEADERS = ["pcg_internal.h", "device.cuh", "kernels.cuh", "handle.cuh", "kernel_table.cuh", "solve_graph.cuh"]


def _sources():
    return ([os.path.join(CSRC, f) for f in CU_SOURCES + CPP_SOURCES + HEADERS]
            + [os.path.join(ROOT, "include", "pcg.h")])


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.exists(s) and os.path.getmtime(s) > t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not needs_build():
        return LIB
    bdir = os.path.join(HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    objs = []
    for f in CPP_SOURCES:
        o = os.path.join(bdir, f + ".o")
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-fast-math",
               "-I", os.path.join(ROOT, "include"), "-c", os.path.join(CSRC, f), "-o", o]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
        objs.append(o)
    cmds = []
    for f in CU_SOURCES:
        o = os.path.join(bdir, f + ".o")
        cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "-I", os.path.join(ROOT, "include"), "-c", os.path.join(CSRC, f), "-o", o]
        if os.environ.get("PCG_PTXAS_VERBOSE"):
            cmd.insert(1, "-Xptxas=-v")
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        cmds.append(cmd)
        objs.append(o)
    # the translation units are independent: compile them side by side
    with ThreadPoolExecutor(max_workers=min(len(cmds), os.cpu_count() or 1)) as pool:
        for f in [pool.submit(subprocess.check_call, c) for c in cmds]:
            f.result()
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [NVCC, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
           "-Xlinker", "-rpath=/usr/local/cuda/lib64", "-lpthread"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
