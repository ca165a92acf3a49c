"""Build the CUDA library libhybrid1d.so for sm_103a (in-tree, no cmake).

The translation units are compiled in parallel with nvcc and linked into
``paper_1508_02892_gb300/_build/libhybrid1d.so``.  Host code is compiled with
``-ffp-contract=off`` so that the host-side derived constants do not depend on
the host CPU (x86 here, Arm on the GPU machines).
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libhybrid1d.so")
SOURCES = ["hyb_electron.cu", "hyb_sort.cu", "hyb_ion.cu", "hyb_field.cu", "hyb_api.cu", "hyb_noalloc.cu",
           "hyb_swarm.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(home, "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _flags():
    # fast single-precision division and square root, and single-precision
    # denormals flushed to zero, so that the approximate functions of the
    # split-mode kernels (log, square root, reciprocal, division) carry no
    # denormal handling: no FP32 quantity of the split path is near 1e-38 (the
    # smallest, a uniform draw, is 6e-8); double precision is unaffected
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "--prec-div=false", "--prec-sqrt=false", "-ftz=true",
                   "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
                   "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    out_dir = BUILD
    lib = LIB
    extra = []
    os.makedirs(out_dir, exist_ok=True)
    headers = [os.path.join(CSRC, "hyb_internal.cuh"), os.path.join(CSRC, "hyb_device.cuh"),
               os.path.join(ROOT, "include", "hybrid1d.h")]
    objs = []
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(out_dir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s, os.path.abspath(__file__)] + headers):
            jobs.append([_nvcc()] + _flags() + extra + ["-c", s, "-o", o])
    if jobs:
        with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            res = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, res):
            if verbose or r.returncode:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode:
                raise RuntimeError("nvcc failed: " + " ".join(cmd))
    if force or jobs or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [_nvcc()] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link failed")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
