"""Builds the CPU oracle's shared library with gcc (plain C11, OpenMP when available)."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lqs_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblqs_oracle.so")


def _openmp_ok() -> bool:
    try:
        r = subprocess.run(["gcc", "-fopenmp", "-x", "c", "-E", "-"], input=b"", capture_output=True)
        return r.returncode == 0
    except OSError:
        return False


def build(force: bool = False) -> str:
    """Compiles the oracle if the library is missing or older than its source."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fcx-limited-range"]
    if _openmp_ok():
        cmd.append("-fopenmp")
    cmd += [SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
