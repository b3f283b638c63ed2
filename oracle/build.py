"""Compile the C oracle into oracle/_liboracle.so (test infrastructure only).

-ffp-contract=off keeps every a*b+c as two rounded IEEE operations on every
host architecture, so the oracle's arithmetic is the expression order written
in iccg_oracle.c.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "iccg_oracle.c"), os.path.join(HERE, "par_leiden.c")]
LIB = os.path.join(HERE, "_liboracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(s) for s in SRCS):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                           "-shared", "-fPIC", "-o", tmp] + SRCS + ["-lm"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
