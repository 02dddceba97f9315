"""Builds libufalcon_gb300.so in-tree (paper_1801_05745_gb300/_build/).

nvcc compiles each CUDA translation unit for sm_103a only; g++ compiles the
host cosmology; the objects are linked into one shared library.  No cmake,
no torch extension machinery: the library has a plain C ABI.

build(checked=True) makes libufalcon_gb300_checked.so (objects in
_build/checked/): the same library compiled with -DUFC_CHECKED, whose
kernels test their computed indices before each access (ufc_synchronize
reports a failed test as UFC_ERR_INTERNAL).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libufalcon_gb300.so")
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU = ["bin.cu", "stats.cu", "sht.cu", "capi.cu"]
CPP = ["cosmo.cpp", "welford.cpp"]
HEADERS = ["common.cuh", "pixel.cuh", "ctx.h"]


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd: list[str]) -> None:
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("compile failed: " + " ".join(cmd))


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    bdir = os.path.join(BUILD, "checked") if checked else BUILD
    lib = os.path.join(BUILD, "libufalcon_gb300_checked.so") if checked else LIB
    defs = ["-DUFC_CHECKED"] if checked else []
    os.makedirs(bdir, exist_ok=True)
    include = os.path.join(os.path.dirname(HERE), "include", "ufalcon.h")
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [include]
    jobs = []
    objs = []
    for f in CU:
        src = os.path.join(CSRC, f)
        obj = os.path.join(bdir, f + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + hdrs):
            jobs.append([NVCC, *ARCH, *defs, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler",
                         "-fPIC", "-Xptxas", "-v" if verbose else "-O3", "-c", src, "-o", obj])
    for f in CPP:
        src = os.path.join(CSRC, f)
        obj = os.path.join(bdir, f + ".o")
        objs.append(obj)
        if force or _stale(obj, [src, include]):
            jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off",
                         "-fno-fast-math", "-c", src, "-o", obj])
    with cf.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        list(ex.map(_run, jobs))
    if force or jobs or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        _run([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                checked="--checked" in sys.argv))
