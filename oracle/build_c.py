"""Compile the oracle's C step (oracle/cstep.c) into oracle/_build/libue_oracle.so.

Test infrastructure: the compiled oracle times the CPU baseline on the host cores.  gcc -O3
with OpenMP; without OpenMP (no libgomp) it builds single-threaded and says so.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cstep.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libue_oracle.so")


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".{os.getpid()}.tmp"
    base = ["gcc", "-O3", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", SRC, "-o", tmp]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:] + ["-lm"], capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(base + ["-lm"], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle C build failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
