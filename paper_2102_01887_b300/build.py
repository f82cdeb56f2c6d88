"""Build the CUDA library ``libllama.so`` in-tree for sm_103a (B300).

Usage: ``python -m paper_2102_01887_b300.build [--force]``.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
LIB = os.path.join(PKG, "libllama.so")
SOURCES = [os.path.join(PKG, "csrc", f) for f in ("kernels.cu", "llama_host.cu", "llama_static.cu", "sg_gemm.cu", "sg_mlp.cu", "sg_score.cu", "server.cpp")]
DEPS = SOURCES + glob.glob(os.path.join(PKG, "csrc", "*.cuh")) + glob.glob(os.path.join(ROOT, "include", "*.h"))
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2,-Wall", "-shared",
         "-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64",
         "-I" + os.path.join(ROOT, "include")]


def needs_build(out: str = LIB) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in DEPS)


def build(force: bool = False, out: str = LIB, extra: tuple = (), verbose: bool = False) -> str:
    if force or needs_build(out):
        cmd = [NVCC, *ARCH, *FLAGS, *extra, "-o", out, *SOURCES]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.run(cmd, check=True)
    return out


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
