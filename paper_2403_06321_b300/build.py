"""Builds libvbd.so (the C-ABI library of include/vbd.h) in-tree for sm_103a."""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libvbd.so")
SOURCES = ["vbd_kernels.cu", "vbd_collide.cu", "vbd_adjoint.cu", "vbd_host.cpp"]
HEADERS = [os.path.join(CSRC, "vbd_kernels.h"), os.path.join(CSRC, "vbd_geom.cuh"),
           os.path.join(ROOT, "include", "vbd.h")]

NVCC_FLAGS = [
    "-O3", "-std=c++17", "-lineinfo",
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-Xcompiler", "-fPIC,-O2,-fopenmp",
    "-Xptxas", "-v",
]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def build(force: bool = False, verbose: bool = False, defines=()) -> str:
    """Compiles libvbd.so when a source is newer than it (or force).  defines:
    extra -D macros (tuning experiments)."""
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    newest = max(os.path.getmtime(p) for p in srcs + HEADERS + [__file__])
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [_nvcc(), *NVCC_FLAGS, *["-D" + d for d in defines], "-shared", "-cudart", "static",
           "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-o", tmp, *srcs, "-lgomp"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    log = os.path.join(CSRC, "..", "build_ptxas.log")
    with open(log, "w") as f:
        f.write(" ".join(cmd) + "\n" + res.stdout + res.stderr)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError("nvcc failed building libvbd.so")
    if verbose:
        sys.stderr.write(res.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
