"""Build the checker's shared library (libhirace.so) in-tree for sm_103a.

The library is plain C-ABI: CUDA kernels and host code compiled with nvcc,
static CUDA runtime, no PyTorch types.  Each translation unit compiles in
parallel; the link step produces ``paper_2401_04701_gb300/libhirace.so``.
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
LIB = os.path.join(PKG, "libhirace.so")
WORKLOADS_LIB = os.path.join(PKG, "libhirace_workloads.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["hr_kernels.cu", "hr_binned.cu", "hr_api.cu", "hr_fsm.cpp", "hr_noalloc.cu", "hr_shard.cu"]
WORKLOAD_SOURCES = ["hr_workloads.cu"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _compile(src: str, verbose: bool) -> str:
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    cmd = [_nvcc(), "-c", os.path.join(CSRC, src), "-o", obj, "-O3", "-std=c++17", "-lineinfo",
           "-Xcompiler", "-fPIC", "-I", INCLUDE] + ARCH
    if src.endswith(".cu"):
        cmd += ["-Xptxas", "-v"] if verbose else []
    else:
        cmd += ["-x", "cu"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, res.stdout, res.stderr))
    if verbose and res.stderr:
        sys.stderr.write(res.stderr)
    return obj


def _stale() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(WORKLOADS_LIB):
        return True
    t = min(os.path.getmtime(LIB), os.path.getmtime(WORKLOADS_LIB))
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + \
           [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)] + [__file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    every = SOURCES + WORKLOAD_SOURCES
    with cf.ThreadPoolExecutor(len(every)) as ex:
        objs = dict(zip(every, ex.map(lambda s: _compile(s, verbose), every)))
    for lib, srcs in ((LIB, SOURCES), (WORKLOADS_LIB, WORKLOAD_SOURCES)):
        tmp = lib + ".tmp%d" % os.getpid()
        cmd = [_nvcc(), "-shared", "-o", tmp] + [objs[s] for s in srcs] + ARCH + \
              ["-cudart", "static", "-Xcompiler", "-fPIC"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (res.stdout, res.stderr))
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
