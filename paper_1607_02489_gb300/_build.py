"""Compile the C-ABI library libemin_amg.so for sm_103a, in-tree.

The host setup (csrc/setup.cpp) is built with -ffp-contract=off so that the
integer decisions it takes from floating point do not change with the
machine's fused multiply-add; the CUDA sources are compiled for
compute_103a / sm_103a only.  The translation units compile in parallel.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libemin_amg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libemin_amg.so")


def _sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))
            if f.endswith((".cu", ".cuh", ".cpp", ".hpp"))] + [os.path.join(os.path.dirname(HERE), "include", "emin_amg.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    """Build (if stale) and return the path of libemin_amg.so."""
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off", "-I", CSRC]
    jobs = [
        ([nvcc, "-x", "c++", "-c", os.path.join(CSRC, "setup.cpp"), "-o", os.path.join(BUILD, "setup.o")] + common),
        ([nvcc, "-x", "c++", "-c", os.path.join(CSRC, "checkpoint.cpp"), "-o", os.path.join(BUILD, "checkpoint.o")]
         + common),
        ([nvcc, "-c", os.path.join(CSRC, "solver.cu"), "-o", os.path.join(BUILD, "solver.o")] + ARCH + common),
        ([nvcc, "-c", os.path.join(CSRC, "server.cu"), "-o", os.path.join(BUILD, "server.o")] + ARCH + common),
        ([nvcc, "-c", os.path.join(CSRC, "gpu_setup.cu"), "-o", os.path.join(BUILD, "gpu_setup.o")] + ARCH + common),
        ([nvcc, "-c", os.path.join(CSRC, "vcycle_inst.cu"), "-DEMIN_VCYCLE_DOUBLE", "-o",
          os.path.join(BUILD, "vcycle_f64.o")] + ARCH + common),
        ([nvcc, "-c", os.path.join(CSRC, "vcycle_inst.cu"), "-o", os.path.join(BUILD, "vcycle_f32.o")] + ARCH + common),
    ]
    procs = [subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True) for cmd in jobs]
    errors = []
    for cmd, p in zip(jobs, procs):
        out, _ = p.communicate()
        if verbose and out:
            sys.stdout.write(out)
        if p.returncode != 0:
            errors.append(" ".join(cmd) + "\n" + out)
    if errors:
        raise RuntimeError("building libemin_amg.so failed:\n" + "\n".join(errors))
    objs = [os.path.join(BUILD, o) for o in ("setup.o", "checkpoint.o", "solver.o", "server.o", "gpu_setup.o",
                                             "vcycle_f64.o", "vcycle_f32.o")]
    tmp = LIB + ".tmp"
    link = [nvcc, "-shared", "-o", tmp] + objs + ARCH
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("linking libemin_amg.so failed:\n" + r.stdout)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
