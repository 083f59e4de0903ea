"""Compile the oracle's C loops into ``oracle/_liboracle.so`` with gcc.

Test infrastructure: the oracle is compiled FP64, without FMA contraction
(``-ffp-contract=off``), with OpenMP when the compiler supports it.
"""

from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sv_oracle.c")
LIB = os.path.join(HERE, "_liboracle.so")


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", SRC]
    tmp = LIB + f".tmp{os.getpid()}"
    for extra in (["-fopenmp"], []):
        cmd = base[:1] + extra + base[1:] + ["-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, LIB)
            if verbose:
                print(" ".join(cmd))
            return LIB
        if verbose:
            print(r.stderr, file=sys.stderr)
    raise RuntimeError("oracle: gcc failed to build sv_oracle.c:\n" + r.stderr)


if __name__ == "__main__":
    print(build(force=True, verbose=True))
