"""Compiles the oracle's C part (exact_pairs.c) into oracle/liboracle_pairs.so.

TEST INFRASTRUCTURE ONLY: the library is the CPU oracle's exact pair
enumeration; nothing on the product path loads it.  gcc with OpenMP,
plain -O2 (no machine-specific flags: the same source builds on x86 and
Arm hosts).  Rebuilds only when the source is newer than the library.
"""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "exact_pairs.c")
LIB = os.path.join(HERE, "liboracle_pairs.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler for the oracle's exact_pairs.c")
    tmp = LIB + ".tmp"
    r = subprocess.run([cc, "-O2", "-std=c99", "-fopenmp", "-shared", "-fPIC", SRC, "-o", tmp, "-lm"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"oracle C build failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
