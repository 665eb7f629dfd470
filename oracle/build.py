"""Compile the oracle's plain-C parts (test infrastructure only).

``python -m oracle.build`` or ``oracle.build.build()`` writes
``oracle/_build/liboracle.so`` with gcc.  No optimisation flags beyond -O2 and
nothing machine-specific, so the same source builds on x86_64 and aarch64.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "liboracle.so")
SOURCES = [os.path.join(HERE, "greedy_colour.c"), os.path.join(HERE, "clearance.c")]


def build(force=False):
    os.makedirs(BUILD_DIR, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in SOURCES)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp] + SOURCES)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
