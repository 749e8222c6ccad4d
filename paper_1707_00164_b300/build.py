"""Build libgofmm.so in-tree (paper_1707_00164_b300/lib/) for sm_103a.

Host C++ (compression, C ABI) is compiled with g++ -O3 -fopenmp
-ffp-contract=off; the CUDA sources with nvcc for arch sm_103a only; the
shared library links the CUDA runtime statically.  Usage:
    python paper_1707_00164_b300/build.py [--force]
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "lib")
LIB = os.path.join(OUT_DIR, "libgofmm.so")
OBJ_DIR = os.path.join(ROOT, "_build")
INCLUDE = os.path.join(ROOT, "include")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CXX_SOURCES = ["compress.cpp", "abi.cpp", "tune.cpp"]
CU_SOURCES = ["eval.cu", "eval_tc.cu", "eval_static.cu", "engine.cu", "sample.cu"]


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "gofmm.h"))
    files.append(os.path.abspath(__file__))
    return files


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd):
    print(" ".join(cmd), flush=True)
    subprocess.check_call(cmd)


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(OBJ_DIR, exist_ok=True)
    deps = _deps()
    if not force and not _stale(LIB, deps):
        return LIB
    objs = []
    for src in CXX_SOURCES:
        obj = os.path.join(OBJ_DIR, src + ".o")
        _run(["g++", "-std=c++17", "-O3", "-fPIC", "-fopenmp", "-ffp-contract=off", "-Wall",
              "-I", INCLUDE, "-I", "/usr/local/cuda/include", "-c", os.path.join(CSRC, src), "-o", obj])
        objs.append(obj)
    for src in CU_SOURCES:
        obj = os.path.join(OBJ_DIR, src + ".o")
        cmd = [NVCC, "-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC",
               "-I", INCLUDE, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose_ptxas:
            cmd[1:1] = ["-Xptxas", "-v"]
        _run(cmd)
        objs.append(obj)
    tmp = LIB + ".tmp"
    _run([NVCC, "-shared", *ARCH, "-o", tmp, *objs, "-Xcompiler", "-fopenmp", "-cudart", "static"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose_ptxas="--ptxas" in sys.argv)
