"""Builds librmb.so (the CUDA library behind include/rmb.h) in-tree for sm_103a."""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "librmb.so")
# one translation unit per kernel family, compiled in parallel and linked into one library
SOURCES = [os.path.join(CSRC, f) for f in ("rmb.cu", "rmb_csr.cu", "rmb_dense.cu", "rmb_small.cu")]
DEPS = SOURCES + [os.path.join(CSRC, "rmb_core.cuh"), os.path.join(CSRC, "rmb_device.cuh"),
                  os.path.join(ROOT, "include", "rmb.h")]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def compile_cmd(src: str, obj: str, extra=()):
    return [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-I" + os.path.join(ROOT, "include"),
            "-Xcompiler", "-fPIC,-O2", *extra, "-c", "-o", obj, src]


def link_cmd(objs, out: str):
    return [NVCC, *ARCH, "-shared", "-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64", "-o", out, *objs]


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in DEPS):
            return LIB
    extra = ["-Xptxas", "-v"] if verbose else []
    objdir = os.path.join(PKG, "_build")
    os.makedirs(objdir, exist_ok=True)
    objs = [os.path.join(objdir, os.path.basename(src)[:-3] + ".o") for src in SOURCES]
    procs = [subprocess.Popen(compile_cmd(src, obj, extra)) for src, obj in zip(SOURCES, objs)]
    codes = [pr.wait() for pr in procs]
    if any(codes):
        raise subprocess.CalledProcessError(next(c for c in codes if c), "nvcc")
    tmp = LIB + ".tmp"
    subprocess.run(link_cmd(objs, tmp), check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
