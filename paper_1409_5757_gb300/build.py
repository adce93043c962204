"""Compile the CUDA libraries in-tree for sm_103a.

    libefft.so         the transform (csrc/efft.cu; C ABI in include/efft.h)
    libefft_inputs.so  seeded device inputs and norms (csrc/inputs.cu;
                       include/efft_inputs.h), test/benchmark harness only

Both are built with one -gencode (compute_103a -> sm_103a) in parallel; a
library is rebuilt only when one of its sources is newer than the .so.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INC = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-I", INC]

LIBS = {
    "libefft.so": (["efft.cu", "efft_noalloc.cu"],
                   ["efft.cu", "efft_noalloc.cu", "efft_kernels.cuh", "efft_arith.cuh"], ["efft.h"]),
    "libefft_inputs.so": (["inputs.cu"], ["inputs.cu"], ["efft_inputs.h"]),
}


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def lib_path(name: str) -> str:
    return os.path.join(PKG, name)


def _stale(name: str) -> bool:
    out = lib_path(name)
    if not os.path.exists(out):
        return True
    _, deps, hdrs = LIBS[name]
    t = os.path.getmtime(out)
    srcs = [os.path.join(CSRC, d) for d in deps] + [os.path.join(INC, h) for h in hdrs]
    return any(os.path.getmtime(s) > t for s in srcs)


def build(force: bool = False, verbose: bool = False) -> dict:
    """Build both libraries; returns {name: path}."""
    procs = []
    for name, (srcs, _, _) in LIBS.items():
        if not force and not _stale(name):
            continue
        out = lib_path(name)
        tmp = out + ".tmp"
        cmd = [nvcc(), *ARCH, *COMMON, "-o", tmp, *[os.path.join(CSRC, s) for s in srcs]]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((name, out, tmp, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    for name, out, tmp, p in procs:
        log, _ = p.communicate()
        if p.returncode != 0:
            errors.append(f"{name}:\n{log.decode(errors='replace')}")
        else:
            os.replace(tmp, out)
            if verbose and log:
                print(log.decode(errors="replace"))
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    return {name: lib_path(name) for name in LIBS}


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
