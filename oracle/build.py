"""Build the CPU oracle (test infrastructure only) as a shared library.

Compiled with -ffp-contract=off so that every binary32 expression rounds
after each operation, as the oracle's definitions require.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ca_oracle.c")
SRC_SC = os.path.join(HERE, "ca_scorer_oracle.c")
SRC_SC2 = os.path.join(HERE, "ca_scorer2d_oracle.c")
HDR = os.path.join(HERE, "ca_oracle.h")
LIB = os.path.join(HERE, "libca_oracle.so")


def _native_elf(path: str) -> bool:
    """True if `path` is an ELF object for this machine (x86_64 or aarch64)."""
    import platform
    import struct
    try:
        with open(path, "rb") as f:
            head = f.read(20)
    except OSError:
        return False
    if len(head) < 20 or head[:4] != b"\x7fELF":
        return False
    machine = struct.unpack("<H", head[18:20])[0]
    want = {"x86_64": 62, "AMD64": 62, "aarch64": 183, "arm64": 183}.get(platform.machine())
    return want is None or machine == want


def build(force: bool = False) -> str:
    stale = force or not os.path.exists(LIB) or not _native_elf(LIB) or any(
        os.path.getmtime(f) > os.path.getmtime(LIB) for f in (SRC, SRC_SC, SRC_SC2, HDR, __file__))
    if stale:
        tmp = LIB + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-Wall", "-o", tmp, SRC, SRC_SC, SRC_SC2, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
