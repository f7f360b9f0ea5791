"""Builds the in-tree CUDA library ``libsf_gb300.so`` for sm_103a.

Each translation unit in ``csrc/`` is compiled by nvcc in parallel, then
linked into one shared library next to this file. Only the GB300 target is
generated (``-gencode arch=compute_103a,code=sm_103a``). ``debug=True``
builds ``libsf_gb300_debug.so`` instead, with ``-DSF_DEBUG_CHECKS=1``
(shared-memory canaries and index checks in the fused kernels, reported as
SF_ERR_DEBUG_CHECK); the release library has none of them.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libsf_gb300.so")
LIB_DEBUG = os.path.join(HERE, "libsf_gb300_debug.so")
BUILD_DIR = os.path.join(ROOT, "_build")
BUILD_DIR_DEBUG = os.path.join(ROOT, "_build_debug")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def sources():
    """The translation units, the slowest to compile first (adjoint and
    tensor-memory kernels, larger robot buckets)."""
    def cost(f):
        heavy = ("backward" in f) * 2 + ("_tm_" in f) * 2
        n = 0
        for tok in f[:-3].split("_"):
            if tok.startswith("n") and tok[1:].isdigit():
                n = int(tok[1:])
        return (-heavy, -n, f)
    return [os.path.join(CSRC, f) for f in sorted((f for f in os.listdir(CSRC) if f.endswith(".cu")), key=cost)]


def _deps_mtime():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "sf.h"))
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, debug: bool = False) -> str:
    lib = LIB_DEBUG if debug else LIB
    bdir = BUILD_DIR_DEBUG if debug else BUILD_DIR
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime():
        return lib
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    if debug:
        extra += ["-DSF_DEBUG_CHECKS=1"]

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src) + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose or ptxas_info:
            sys.stdout.write(r.stdout + r.stderr)
        return obj

    srcs = sources()
    with ThreadPoolExecutor(max_workers=max(1, min(os.cpu_count() or 1, len(srcs)))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv,
                debug="--debug" in sys.argv))
