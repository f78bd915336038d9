"""Build the CUDA library ``libnwqgb.so`` in-tree for sm_103a (nvcc only).

Each translation unit is compiled in parallel, then linked into one shared
library next to this file.  No torch headers are involved: the library's
interface is the plain C ABI of include/nwqgb.h.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libnwqgb.so")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["sweep_kernels.cu", "expect_kernels.cu", "batch_kernels.cu", "noalloc.cu", "tc_kernels.cu", "probe.cu", "planner.cpp", "tc_plan.cpp", "plan_check.cpp", "jit.cpp", "expect_host.cpp", "abi.cpp", "batch_host.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _flags(src):
    f = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-lineinfo", "-I", os.path.join(ROOT, "include")]
    if src.endswith(".cu"):
        f += ARCH + ["--expt-relaxed-constexpr"]
    else:
        f += ["-x", "c++"]
    return f


def _compile(src):
    obj = os.path.join(BUILD, src + ".o")
    path = os.path.join(CSRC, src)
    deps = [path] + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".hpp", ".cuh"))]
    deps.append(os.path.join(ROOT, "include", "nwqgb.h"))
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(d) for d in deps):
        return obj
    cmd = [NVCC, *_flags(src), "-c", path, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj


def build(verbose=False):
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(_compile, SOURCES))
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(o) for o in objs):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True)
    sys.exit(0)
