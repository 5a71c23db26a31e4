"""Compile the CUDA library in-tree: libcher.so next to this file.

nvcc, one -gencode for sm_103a, the three translation units compiled in
parallel and linked with the static CUDA runtime.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libcher.so")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["cher_kernels.cu", "cher_adjoint.cu", "cher_api.cu", "cher_generator.cu", "cher_pack.cu",
           "cher_tables.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _flags(src: str):
    f = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-lineinfo"] + ARCH
    if not src.endswith(".cu"):
        return f + ["-x", "c++"]
    if os.environ.get("CHER_PTXAS_VERBOSE"):
        f += ["-Xptxas", "-v"]
    if src == "cher_kernels.cu":
        # single-precision division and square root by the hardware
        # approximations (<= 2 ulp); double precision is unaffected and the
        # FP64 yield uses explicitly rounded intrinsics
        f += ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"]
    return f


def _newest_input() -> float:
    paths = [os.path.join(CSRC, s) for s in os.listdir(CSRC)]
    paths.append(os.path.join(HERE, "..", "include", "cher.h"))
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(OUT) and os.path.getmtime(OUT) >= _newest_input():
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, src + ".o")
        cmd = [cc, "-c", os.path.join(CSRC, src), "-o", obj] + _flags(src)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = OUT + ".tmp"
    cmd = [cc, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
