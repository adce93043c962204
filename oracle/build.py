"""Build the CPU oracle (plain C, FP64, OpenMP) as a shared library.

Test infrastructure: the oracle is built here so that tests/, bench.py's
cpu_baseline leg and __graft_entry__.smoke() can load it.  The product
library never links or loads it.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")


def lib_path(mutant: int = 0, outdir: str | None = None) -> str:
    name = "liboracle.so" if mutant == 0 else f"liboracle_mutant{mutant}.so"
    return os.path.join(outdir or HERE, name)


def build(mutant: int = 0, outdir: str | None = None, force: bool = False) -> str:
    """Compile oracle.c (optionally with a planted mistake) and return the .so path."""
    out = lib_path(mutant, outdir)
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= max(os.path.getmtime(SRC),
                                             os.path.getmtime(os.path.join(HERE, "oracle.h")))
            and mutant == 0):
        return out
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-shared", "-fPIC", "-Wall", "-Wextra", "-Wno-unused-parameter",
           f"-DORACLE_MUTANT={int(mutant)}", "-o", out, SRC, "-lm"]
    tmp = out + ".tmp"
    cmd[cmd.index(out)] = tmp
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
