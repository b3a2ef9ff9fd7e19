"""Builds ``lib/libiblbm.so`` in-tree from ``csrc/`` for sm_103a (GB300),
and ``lib/libiblbm_checked.so``, the same sources with the kernels' computed
indices range-checked (-DIBLBM_BOUNDS_CHECK).

CUDA translation units are compiled by nvcc in parallel, host translation
units by g++ (no FMA contraction, so host geometry rounds the same on x86 and
Arm), and the objects are linked into one shared library with a static CUDA
runtime.  Objects go to ``_build/`` beside the package; both are ignored by
git.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJ = os.path.join(HERE, "_build")
LIB_DIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIB_DIR, "libiblbm.so")

CUDA_UNITS = ["lbm.cu", "ib.cu", "taylor.cu", "adjoint.cu"]
HOST_UNITS = ["capi.cpp", "mesh.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home() -> str:
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _sources():
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hdrs.append(os.path.join(INCLUDE, "iblbm.h"))
    return hdrs


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _variant_jobs(variant: str, cuda: str, force: bool):
    """(compile jobs, objects, library) of one variant: "" the library,
    "checked" the bounds-checked build of the same sources."""
    nvcc = os.path.join(cuda, "bin", "nvcc")
    obj_dir = os.path.join(OBJ, variant) if variant else OBJ
    lib = os.path.join(LIB_DIR, f"libiblbm_{variant}.so" if variant else "libiblbm.so")
    extra = ["-DIBLBM_BOUNDS_CHECK"] if variant == "checked" else []
    os.makedirs(obj_dir, exist_ok=True)
    hdrs = _sources()
    jobs, objs = [], []
    for u in CUDA_UNITS:
        src = os.path.join(CSRC, u)
        obj = os.path.join(obj_dir, u + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + hdrs):
            jobs.append([nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", *extra,
                         "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj])
    for u in HOST_UNITS:
        src = os.path.join(CSRC, u)
        obj = os.path.join(obj_dir, u + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + hdrs):
            jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", *extra,
                         "-I", INCLUDE, "-I", CSRC, "-I", os.path.join(cuda, "include"),
                         "-c", src, "-o", obj])
    return jobs, objs, lib


def build(force: bool = False, verbose: bool = False, variants=("", "checked")) -> str:
    """Compiles every translation unit of every variant in parallel, then
    links each variant's library; returns the path of the main library."""
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(OBJ, exist_ok=True)
    os.makedirs(LIB_DIR, exist_ok=True)
    plans = [(_variant_jobs(v, cuda, force)) for v in variants]
    jobs = [j for p in plans for j in p[0]]
    procs = [(cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)) for cmd in jobs]
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode:
            failed.append(" ".join(cmd))
    if failed:
        raise RuntimeError("compilation failed:\n" + "\n".join(failed))
    for vjobs, objs, lib in plans:
        if force or vjobs or _stale(lib, objs):
            tmp = lib + f".tmp{os.getpid()}"
            cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
            r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
            if r.returncode:
                sys.stderr.write(r.stdout.decode(errors="replace"))
                raise RuntimeError("link failed: " + " ".join(cmd))
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
