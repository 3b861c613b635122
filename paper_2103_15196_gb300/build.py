"""Builds the in-tree CUDA library ``_lib/libswe.so`` for sm_103a with nvcc.

Three translation units compiled in parallel: the FP32 kernels (fast-math
intrinsics), the FP64 kernels (``--fmad=false``: every operation rounds as
written, matching the FP64 CPU oracle's order), and the C-ABI host code.
The CUDA runtime is linked statically, so the library needs only the driver.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libswe.so")
# the checked variant (-DSWE_CHECKED): every global index of the step kernel
# is tested against its buffer; built on demand by the tests
LIB_CHECKED = os.path.join(OUT_DIR, "libswe_checked.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", SRC] + ARCH
UNITS = {
    "swe_f32.cu": ["--use_fast_math"],
    "swe_f64.cu": ["--fmad=false"],
    "swe_capi.cu": [],
    "swe_noalloc.cu": [],
    "swe_ensemble.cu": ["--use_fast_math"],
    "nn_kernels.cu": [],
}


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return p


def _sources():
    return [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".cu", ".cuh", ".h"))] + \
           [os.path.join(INCLUDE, "swe.h")]


def up_to_date(checked: bool = False) -> bool:
    lib = LIB_CHECKED if checked else LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False, extra=(), checked: bool = False) -> str:
    lib = LIB_CHECKED if checked else LIB
    if not force and up_to_date(checked):
        return lib
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    extra = list(extra) + (["-DSWE_CHECKED"] if checked else [])

    def compile_one(name):
        obj = os.path.join(OUT_DIR, name.replace(".cu", "_checked.o" if checked else ".o"))
        cmd = [cc, "-c", os.path.join(SRC, name), "-o", obj] + COMMON + UNITS[name] + list(extra)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = lib + f".{os.getpid()}.tmp"
    r = subprocess.run([cc, "-shared", "-o", tmp] + objs + ARCH, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else [])
    print(LIB)
