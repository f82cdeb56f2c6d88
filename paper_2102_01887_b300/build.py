"""Build the CUDA library ``libllama.so`` in-tree for sm_103a (B300).

Every source is compiled to its own object (in parallel, under ``_build/``),
then the objects are linked into the shared library.

Usage: ``python -m paper_2102_01887_b300.build [--force]``.
"""
from __future__ import annotations

import glob
import hashlib
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
LIB = os.path.join(PKG, "libllama.so")
CHECK_LIB = os.path.join(PKG, "libllama_check.so")  # bounds checks that set bits (-DLLAMA_CHECK)
OBJ_DIR = os.path.join(ROOT, "_build")
SOURCES = [os.path.join(PKG, "csrc", f) for f in ("kernels.cu", "llama_host.cu", "llama_static.cu", "sg_gemm.cu", "sg_mlp.cu", "sg_score.cu", "server.cpp", "alu_peak.cu", "count_rate.cu", "loop.cu", "loop_arrivals.cpp", "stragglers.cpp")]
HEADERS = glob.glob(os.path.join(PKG, "csrc", "*.cuh")) + glob.glob(os.path.join(PKG, "csrc", "*.h")) + \
    glob.glob(os.path.join(ROOT, "include", "*.h"))
DEPS = SOURCES + HEADERS
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2,-Wall",
          "-I" + os.path.join(ROOT, "include")]
LDFLAGS = ["-shared", "-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64"]


def needs_build(out: str = LIB) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in DEPS)


def _object(src: str, extra: tuple) -> str:
    tag = hashlib.sha256(" ".join(extra).encode()).hexdigest()[:8]
    return os.path.join(OBJ_DIR, f"{os.path.basename(src)}.{tag}.o")


def _compile(src: str, extra: tuple, verbose: bool) -> str:
    obj = _object(src, extra)
    newest_dep = max(os.path.getmtime(d) for d in [src] + HEADERS)
    if os.path.exists(obj) and os.path.getmtime(obj) > newest_dep:
        return obj
    cmd = [NVCC, *ARCH, *CFLAGS, *extra, "-c", "-o", obj, src]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    return obj


def build(force: bool = False, out: str = LIB, extra: tuple = (), verbose: bool = False) -> str:
    """Compile (when a source or header is newer than ``out``) and link ``out``.
    ``extra`` adds compiler flags (for instance ``-DLLAMA_CHECK``)."""
    if force or needs_build(out):
        os.makedirs(OBJ_DIR, exist_ok=True)
        if force:
            for src in SOURCES:
                obj = _object(src, tuple(extra))
                if os.path.exists(obj):
                    os.remove(obj)
        with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
            objs = list(ex.map(lambda s: _compile(s, tuple(extra), verbose), SOURCES))
        cmd = [NVCC, *ARCH, *LDFLAGS, "-o", out + ".tmp", *objs]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.run(cmd, check=True)
        os.replace(out + ".tmp", out)  # a process that has the old library mapped keeps it
    return out


def build_check(force: bool = False, verbose: bool = False) -> str:
    """The checked build, libllama_check.so (-DLLAMA_CHECK)."""
    return build(force=force, out=CHECK_LIB, extra=("-DLLAMA_CHECK",), verbose=verbose)


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    if "--check" in sys.argv:
        build_check(force="--force" in sys.argv, verbose=True)
