"""Build the CUDA library libmisr.so in-tree for sm_103a with nvcc."""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libmisr.so")
LIB_CHECK = os.path.join(PKG, "libmisr_check.so")   # the bounds-checked variant (MISR_BOUNDS_CHECK)
SOURCES = [os.path.join(CSRC, f) for f in ("misr_api.cu", "misr_batch.cu", "misr_server.cu")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h", ".cu"))] + \
    [os.path.join(INCLUDE, "misr.h")]
NVCC_FLAGS = ["-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
              "-Xcompiler", "-fPIC", "-shared", "-Xptxas", "-v", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Build libmisr.so, or with checked=True the bounds-checked libmisr_check.so."""
    lib = LIB_CHECK if checked else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= max(os.path.getmtime(d) for d in DEPS):
        return lib
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nvcc(), *NVCC_FLAGS, *(["-DMISR_BOUNDS_CHECK"] if checked else []), "-I", INCLUDE, "-I", CSRC, "-o", tmp,
           *SOURCES]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if verbose or r.returncode != 0:
        sys.stdout.write(r.stdout)
        sys.stderr.write(r.stderr)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv)
