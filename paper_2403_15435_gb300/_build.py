"""Build libgeoflood.so in-tree with nvcc for sm_103a.

Each translation unit compiles in parallel; the FP64 kernel units use
-fmad=false so that products and sums round exactly as written.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgeoflood.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

# (source, extra flags)
SOURCES = [
    ("gf_step.cu", ["-fmad=false"]),
    # FP32 kernels: approximate single-precision division and square root
    # (a few ulp; the FP32 path is held to absolute tolerances, and a lake at
    # rest still gives exactly zero waves), denormals flushed to zero
    ("gf_step32.cu", ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"]),
    ("gf_amr.cu", ["-fmad=false"]),
    ("gf_cnn.cu", []),
    ("gf_forest.cpp", []),
    # host FP64 that must round as the device does (the tag kernel's box
    # test): no contraction into fused multiply-adds
    ("gf_api.cpp", ["-Xcompiler", "-ffp-contract=off"]),
]
HEADERS = ["gf_internal.h", "gf_solver.cuh", "gf_forest.h", "gf_step_kernel.cuh"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"),
                 "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgeoflood.so")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s, _ in SOURCES]
    deps += [os.path.join(CSRC, h) for h in HEADERS]
    deps += [os.path.join(ROOT, "include", "geoflood.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-I" + os.path.join(ROOT, "include")]
    procs = []
    objs = []
    for src, extra in SOURCES:
        obj = os.path.join(BUILD, src.replace(".", "_") + ".o")
        cmd = [cc] + common + extra + ["-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"] if verbose else []
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                            stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode:
            failed.append(src)
    if failed:
        raise RuntimeError("nvcc failed for: " + ", ".join(failed))
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.check_call([cc] + ARCH + ["-shared", "-o", tmp] + objs)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
