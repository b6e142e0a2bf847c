"""Builds libges (the CUDA library behind include/ges.h) for sm_103a, in-tree.

Translation units are compiled in parallel with nvcc and linked into
``paper_2402_10128_gb300/_build/libges.so`` (static CUDA runtime).  Objects are
reused when newer than every source and header.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "libges.so")
SOURCES = ["preprocess.cu", "sort.cu", "raster.cu", "api.cu", "serve.cu", "noalloc.cu", "loss.cu", "train.cu", "mixture1d.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"),
                 os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found (set NVCC or CUDA_HOME)")


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "ges.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def build(verbose: bool = False, force: bool = False, extra_flags=()) -> str:
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    dep = _deps_mtime()
    objs = []
    jobs = []
    for src in SOURCES:
        obj = os.path.join(OUT, src.replace(".cu", ".o"))
        objs.append(obj)
        if force or not os.path.exists(obj) or os.path.getmtime(obj) < dep:
            cmd = [nvcc, *ARCH, *FLAGS, *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj]
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(run, jobs))
    if jobs or force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + f".tmp{os.getpid()}"
        run([nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", *objs, "-o", tmp, "-lpthread", "-ldl", "-lrt"])
        os.replace(tmp, LIB)
    return LIB


MICROBENCH = os.path.join(OUT, "sfu_rates")


def build_microbench() -> str:
    """The SFU-rate microbenchmark (paper_2402_10128_gb300/microbench/sfu_rates.cu)."""
    os.makedirs(OUT, exist_ok=True)
    src = os.path.join(PKG, "microbench", "sfu_rates.cu")
    if not os.path.exists(MICROBENCH) or os.path.getmtime(MICROBENCH) < os.path.getmtime(src):
        tmp = MICROBENCH + f".tmp{os.getpid()}"
        r = subprocess.run([_nvcc(), *ARCH, "-O3", src, "-o", tmp], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for the SFU microbenchmark:\n" + r.stdout + r.stderr)
        os.replace(tmp, MICROBENCH)
    return MICROBENCH


if __name__ == "__main__":
    print(build(verbose=True))
