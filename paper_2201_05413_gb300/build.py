"""Builds the CUDA library libgbpcg.so in-tree for sm_103a (nvcc, no cmake).

Translation units compile in parallel into ``_build/``; the shared library
links the CUDA runtime statically.  ``build()`` recompiles only what changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
# GBPCG_NVCC_DEFINES: extra -D options for experiments (a build of its own
# objects, linked into the same library path)
DEFINES = os.environ.get("GBPCG_NVCC_DEFINES", "").split()
OUT_DIR = os.path.join(HERE, "_build" + ("_" + "_".join(d.lstrip("-D").replace("=", "") for d in DEFINES)
                                         if DEFINES else ""))
LIB = os.path.join(HERE, "libgbpcg.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "-I", os.path.join(ROOT, "include")] + ARCH + DEFINES


def _deps(src):
    deps = [src, os.path.join(ROOT, "include", "gbpcg.h")]
    deps += glob.glob(os.path.join(CSRC, "*.cuh"))
    return deps


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def _compile(src):
    obj = os.path.join(OUT_DIR, os.path.basename(src)[:-3] + ".o")
    if _stale(obj, _deps(src)):
        tmp = obj + f".tmp{os.getpid()}"
        r = subprocess.run([NVCC] + FLAGS + ["-c", src, "-o", tmp], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, obj)
    return obj


def build(verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(_compile, srcs))
    if _stale(LIB, objs) or DEFINES:
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [NVCC] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True)
