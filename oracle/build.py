"""Build the CPU oracle (test infrastructure only) as a shared library.

Compiled with -ffp-contract=off so that every binary32 expression rounds
after each operation, as the oracle's definitions require.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ca_oracle.c")
HDR = os.path.join(HERE, "ca_oracle.h")
LIB = os.path.join(HERE, "libca_oracle.so")


def build(force: bool = False) -> str:
    stale = force or not os.path.exists(LIB) or any(
        os.path.getmtime(f) > os.path.getmtime(LIB) for f in (SRC, HDR, __file__))
    if stale:
        tmp = LIB + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-Wall", "-o", tmp, SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
