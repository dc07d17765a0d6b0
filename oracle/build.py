"""Compile the FP64 CPU oracle (``spo.c``) into ``oracle/libspo.so``.

Test infrastructure: the oracle is the independent reference the CUDA path
is checked against; building it is not using it.  Plain ``gcc -O3`` with
OpenMP, no machine-specific flags, so the same source builds on x86-64 and
aarch64 hosts.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "spo.c")
HDR = os.path.join(HERE, "spo.h")
LIB = os.path.join(HERE, "libspo.so")


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in (SRC, HDR))


def build(force: bool = False) -> str:
    if force or needs_build():
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-std=c99", "-O3", "-fPIC", "-shared", "-fopenmp", "-Wall",
               "-o", tmp, SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
