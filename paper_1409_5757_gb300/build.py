"""Compile the CUDA libraries in-tree for sm_103a.

    libefft.so         the transform (csrc/efft.cu plans and execution,
                       efft_tune.cu autotuner, efft_batch.cu batches,
                       efft_real.cu real-data transforms,
                       efft_mix.cu N = M * 2^e passes,
                       efft_fx_df2.cu / efft_fx_f32.cu pass kernels,
                       efft_noalloc.cu; C ABI in include/efft.h)
    libefft_inputs.so  seeded device inputs and norms (csrc/inputs.cu;
                       include/efft_inputs.h), test/benchmark harness only

Every translation unit is compiled to an object with one -gencode
(compute_103a -> sm_103a), all in parallel, then linked; a library is
rebuilt only when one of its sources or headers is newer than the .so.
Objects go to _build/ (not tracked).
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
OBJ = os.path.join(ROOT, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INC]

# library -> (translation units, headers they depend on)
LIBS = {
    "libefft.so": (["efft.cu", "efft_tune.cu", "efft_batch.cu", "efft_real.cu", "efft_mix.cu", "efft_fx_df2.cu",
                    "efft_fx_f32.cu", "efft_noalloc.cu"],
                   ["efft_kernels.cuh", "efft_arith.cuh", "efft_mix.cuh", "efft_fx32.cuh", "efft_host.h"], ["efft.h"]),
    "libefft_inputs.so": (["inputs.cu"], [], ["efft_inputs.h"]),
}


def nvcc() -> str:
    return shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"


def lib_path(name: str) -> str:
    return os.path.join(PKG, name)


def _stale(name: str) -> bool:
    out = lib_path(name)
    if not os.path.exists(out):
        return True
    srcs, hdrs, incs = LIBS[name]
    t = os.path.getmtime(out)
    deps = [os.path.join(CSRC, d) for d in srcs + hdrs] + [os.path.join(INC, h) for h in incs]
    return any(os.path.getmtime(s) > t for s in deps)


def build(force: bool = False, verbose: bool = False) -> dict:
    """Build both libraries; returns {name: path}."""
    os.makedirs(OBJ, exist_ok=True)
    todo = [name for name in LIBS if force or _stale(name)]
    procs = []
    for name in todo:
        for src in LIBS[name][0]:
            obj = os.path.join(OBJ, src.replace(".cu", f".{os.getpid()}.o"))
            cmd = [nvcc(), *ARCH, *COMMON, "-c", "-o", obj, os.path.join(CSRC, src)]
            if verbose:
                print(" ".join(cmd), flush=True)
            procs.append((name, src, obj, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    objs = {name: [] for name in todo}
    for name, src, obj, p in procs:
        log, _ = p.communicate()
        if p.returncode != 0:
            errors.append(f"{src}:\n{log.decode(errors='replace')}")
        else:
            objs[name].append(obj)
            if verbose and log:
                print(log.decode(errors="replace"))
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    for name in todo:
        out = lib_path(name)
        tmp = out + f".{os.getpid()}.tmp"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs[name]]
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        for o in objs[name]:
            try:
                os.remove(o)
            except OSError:
                pass
        if r.returncode != 0:
            raise RuntimeError(f"link of {name} failed:\n{r.stdout.decode(errors='replace')}")
        os.replace(tmp, out)
    return {name: lib_path(name) for name in LIBS}


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
