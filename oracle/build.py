"""Compile the oracle's C part (integrals.c) into oracle/liboracle.so.

ORACLE -- test infrastructure only (tests, smoke check, benchmark CPU
baseline).  Built with plain gcc; OpenMP is used when the compiler has it.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "integrals.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False, verbose: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-D_GNU_SOURCE", SRC, "-o", tmp, "-lm"]
    for extra in (["-fopenmp"], []):
        cmd = base[:1] + extra + base[1:]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, LIB)
            if verbose:
                print(" ".join(cmd))
            return LIB
    sys.stderr.write(r.stderr)
    raise RuntimeError("could not compile the oracle: %s" % " ".join(base))


if __name__ == "__main__":
    print(build(force=True, verbose=True))
