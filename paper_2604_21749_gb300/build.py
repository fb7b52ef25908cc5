"""Compiles the CUDA library (csrc/*.cu -> _build/libcurast.so) for sm_103a.

The translation units are compiled in parallel with nvcc and linked into one
shared library exporting the C ABI of include/curast.h.  Every kernel is
built with --fmad=false and host code with -ffp-contract=off; the kernels
also use explicitly rounded intrinsics, so no multiply-add is ever fused.
"""
from __future__ import annotations

import os
import platform
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
SOURCES = ["raster.cu", "shade.cu", "runtime.cu", "static_render.cu", "compress.cu"]
HEADERS = ["device.cuh", "internal.h", "stage1.cuh", "stage1_win.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("CUDACXX"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    raise RuntimeError("nvcc not found")


def lib_path() -> str:
    return os.path.join(BUILD, f"libcurast_{platform.machine()}.so")


def _stale(out: str) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(INCLUDE, "curast.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build_library(force: bool = False, verbose: bool = False) -> str:
    out = lib_path()
    if not force and not _stale(out):
        return out
    os.makedirs(BUILD, exist_ok=True)
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "--fmad=false", "-Xcompiler", "-fPIC",
                     "-Xcompiler", "-ffp-contract=off", "-I", INCLUDE, "-I", CSRC, "-Xptxas", "-v"]
    procs, objs = [], []
    for src in SOURCES:
        obj = os.path.join(BUILD, f"{os.path.splitext(src)[0]}_{platform.machine()}.o")
        log = open(obj + ".log", "w")
        cmd = [nvcc()] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        procs.append((subprocess.Popen(cmd, stdout=log, stderr=subprocess.STDOUT), log, obj, cmd))
        objs.append(obj)
    failed = []
    for p, log, obj, cmd in procs:
        rc = p.wait()
        log.close()
        if rc != 0:
            failed.append((obj, cmd))
    if failed:
        msg = []
        for obj, cmd in failed:
            msg.append(" ".join(cmd) + "\n" + open(obj + ".log").read())
        raise RuntimeError("nvcc failed:\n" + "\n".join(msg))
    if verbose:
        for obj in objs:
            sys.stdout.write(open(obj + ".log").read())
    tmp = out + f".tmp{os.getpid()}"
    cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build_library(force="--force" in sys.argv, verbose="-v" in sys.argv))
