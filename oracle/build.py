"""Compile the FP64 CPU oracle (test infrastructure only).

The oracle is plain C built with the host gcc.  It is rebuilt when the shared
object is missing or older than its source.  OpenMP is used when the compiler
supports it (the split is over independent output rows and changes no
arithmetic); otherwise the build falls back to a single-threaded object.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ssim_oracle.c")
LIB = os.path.join(HERE, "libssim_oracle.so")


def build_oracle(force: bool = False, verbose: bool = False) -> str:
    """Build ``libssim_oracle.so`` next to its source and return its path."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
            SRC, "-o", LIB + ".tmp", "-lm"]
    for extra in (["-fopenmp"], []):
        cmd = base[:2] + extra + base[2:]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        if r.returncode == 0:
            os.replace(LIB + ".tmp", LIB)
            return LIB
    raise RuntimeError("oracle build failed:\n" + r.stderr)


if __name__ == "__main__":
    print(build_oracle(force="--force" in sys.argv, verbose=True))
