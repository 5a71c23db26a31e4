"""Compile the CUDA library in-tree: libcher.so next to this file.

nvcc, one -gencode for sm_103a, the translation units compiled in parallel
and linked with the static CUDA runtime.  With debug=True (or CHER_DEBUG=1
in the environment) the bounds-checked variant libcher_debug.so: every
kernel index is checked before its access, a failed check sets a bit of
stats[CHER_STAT_DEBUG] (cher_sync_status then reports CHER_EBOUNDS) and
the access is moved inside the array; nothing traps.
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
OUT_DEBUG = os.path.join(HERE, "libcher_debug.so")
BUILD_DEBUG = os.path.join(HERE, "_build_debug")


def debug_requested() -> bool:
    return os.environ.get("CHER_DEBUG", "") == "1"
SOURCES = ["cher_kernels.cu", "cher_adjoint.cu", "cher_api.cu", "cher_generator.cu", "cher_pack.cu",
           "cher_tables.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _flags(src: str, debug: bool = False):
    f = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-lineinfo"] + ARCH
    if debug:
        f += ["-DCHER_DEBUG"]
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


def build(force: bool = False, verbose: bool = False, debug: bool | None = None) -> str:
    if debug is None:
        debug = debug_requested()
    out, bdir = (OUT_DEBUG, BUILD_DEBUG) if debug else (OUT, BUILD)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= _newest_input():
        return out
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(bdir, src + ".o")
        cmd = [cc, "-c", os.path.join(CSRC, src), "-o", obj] + _flags(src, debug)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = out + ".tmp"
    cmd = [cc, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                debug=True if "--debug" in sys.argv else None))
