"""Build the native library ``libscylla.so`` in-tree for sm_103a (GB300).

The CUDA translation unit is compiled by nvcc for ``-gencode arch=compute_103a,
code=sm_103a``; the host C++ units by g++ with ``-ffp-contract=off`` so the
rounding of the host rounding step is exactly as written.  Units compile in
parallel; the result is linked by nvcc with the static CUDA runtime.

Usage: ``python -m paper_2307_03466_gb300.build`` (or ``build()`` from Python).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libscylla.so")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["kernels.cu", "fanout.cu", "noalloc.cu", "transpose.cu", "setup.cu", "propagate.cu", "infeas.cu"]
CPP_SOURCES = ["lp.cpp", "fixprop.cpp", "pump.cpp", "batch.cpp", "fanout.cpp", "certify.cpp"]


def _sources():
    return [os.path.join(CSRC, f) for f in CU_SOURCES + CPP_SOURCES] + \
        [os.path.join(CSRC, "internal.h"), os.path.join(CSRC, "lp_handle.h"), os.path.join(CSRC, "device_common.cuh"),
         os.path.join(CSRC, "host_par.h"),
         os.path.join(INCLUDE, "scylla.h")]


def _up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link; returns the library path.  Raises on failure."""
    if not force and _up_to_date():
        return LIB
    if not os.path.exists(NVCC):
        raise RuntimeError(f"nvcc not found at {NVCC}")
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    jobs = []
    objs = []
    for f in CU_SOURCES:
        o = os.path.join(BUILD, f + ".o")
        objs.append(o)
        cmd = [NVCC, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
               "-I", INCLUDE, "-I", CSRC, "-Xptxas", "-warn-spills", "-c", os.path.join(CSRC, f), "-o", o]
        jobs.append(cmd)
    for f in CPP_SOURCES:
        o = os.path.join(BUILD, f + ".o")
        objs.append(o)
        cxx = shutil.which("g++") or "g++"
        cmd = [cxx, "-O2", "-std=c++17", "-fPIC", "-pthread", "-ffp-contract=off", "-Wall", "-Wno-unused-function",
               "-I", INCLUDE, "-I", CSRC, "-I", os.path.join(CUDA_HOME, "include"), "-c",
               os.path.join(CSRC, f), "-o", o]
        jobs.append(cmd)
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True) for c in jobs]
    failed = []
    for c, p in zip(jobs, procs):
        out, _ = p.communicate()
        if verbose and out.strip():
            print(out, file=sys.stderr)
        if p.returncode != 0:
            failed.append((c, out))
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + o for c, o in failed)
        raise RuntimeError("native build failed:\n" + msg)
    tmp = LIB + ".tmp"
    link = [NVCC, "-shared", *ARCH, "-o", tmp, *objs, "-cudart", "static", "-lpthread"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + " ".join(link) + "\n" + r.stdout)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
