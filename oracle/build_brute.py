"""Compiles oracle/brute.c into oracle/libtacaw_brute.so (test infrastructure only)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "brute.c")
LIB = os.path.join(HERE, "libtacaw_brute.so")


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", LIB, SRC, "-lm"])
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
