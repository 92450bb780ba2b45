"""Builds the CPU oracle (oracle.c) into a shared library with gcc.

Test infrastructure: the oracle is the checker of the CUDA path, never part of
it.  ``build()`` writes ``liboracle.so`` beside this file; ``build_mutant(k,
out_dir)`` builds the same source with one planted mistake (see oracle.c) for
the pin-sensitivity tests.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

# -ffp-contract=off keeps every step of the FP64 loop a separate rounding
# (RN(RN(a*b) + s)), so the oracle's result is reproducible.
CFLAGS = ["-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread", "-Wall"]


def _compile(out: str, defines=()) -> str:
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", *CFLAGS, *["-D%s" % d for d in defines], SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    return _compile(LIB)


def build_mutant(k: int, out_dir: str) -> str:
    os.makedirs(out_dir, exist_ok=True)
    return _compile(os.path.join(out_dir, "liboracle_mutant%d.so" % k),
                    defines=["ORACLE_MUTANT=%d" % k])


if __name__ == "__main__":
    print(build(force=True))
