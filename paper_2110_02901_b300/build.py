"""Builds librmb.so (the CUDA library behind include/rmb.h) in-tree for sm_103a."""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "librmb.so")
SOURCES = [os.path.join(CSRC, "rmb.cu")]
DEPS = SOURCES + [os.path.join(CSRC, "rmb_device.cuh"), os.path.join(ROOT, "include", "rmb.h")]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def nvcc_cmd(out: str, extra=()):
    return [NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
            "-I" + os.path.join(ROOT, "include"), "-Xcompiler", "-fPIC,-O2", "-shared",
            "-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64",
            *extra, "-o", out, *SOURCES]


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in DEPS):
            return LIB
    extra = ["-Xptxas", "-v"] if verbose else []
    tmp = LIB + ".tmp"
    subprocess.run(nvcc_cmd(tmp, extra), check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
