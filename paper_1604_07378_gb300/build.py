"""Builds the solver's shared library ``_lib/libhqn.so`` in-tree.

Host C++ (set-up, dense factorisation) is compiled with g++, the CUDA sources
with nvcc for sm_103a only; translation units compile in parallel and the
library is linked with nvcc (static CUDA runtime).  Rebuilds only when a
source is newer than the library.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libhqn.so")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")

CXX_SOURCES = ["setup.cpp", "dense.cpp", "tune.cpp"]
CU_SOURCES = ["kernels.cu", "solve.cu", "api.cu", "noalloc.cu", "peak.cu"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the solver library")


def _sources():
    out = [os.path.join(CSRC, f) for f in CXX_SOURCES + CU_SOURCES]
    out += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".hpp"))]
    out.append(os.path.join(INCLUDE, "hqn.h"))
    return out


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build_library(force: bool = False, verbose: bool = False) -> str:
    """Compiles and links libhqn.so if it is missing or out of date; returns its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(os.path.join(LIBDIR, "obj"), exist_ok=True)
    nvcc = _nvcc()
    objdir = os.path.join(LIBDIR, "obj")
    jobs = []
    for f in CXX_SOURCES:
        o = os.path.join(objdir, f + ".o")
        jobs.append(["g++", "-O3", "-std=c++17", "-fPIC", "-fopenmp", "-I" + INCLUDE, "-c",
                     os.path.join(CSRC, f), "-o", o])
    for f in CU_SOURCES:
        o = os.path.join(objdir, f + ".o")
        jobs.append([nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fopenmp",
                     "-Xptxas", "-v" if verbose else "-O3", "-I" + INCLUDE, "-c",
                     os.path.join(CSRC, f), "-o", o])
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        logs = list(ex.map(_run, jobs))
    if verbose:
        for lg in logs:
            print(lg)
    objs = [os.path.join(objdir, f + ".o") for f in CXX_SOURCES + CU_SOURCES]
    tmp = LIB + ".tmp"
    _run([nvcc, ARCH, "-shared", "-o", tmp] + objs + ["-Xcompiler", "-fopenmp", "-lgomp"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build_library(force="--force" in sys.argv, verbose="-v" in sys.argv))
