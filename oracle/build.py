"""Build the CPU oracle shared library (test infrastructure only).

    python oracle/build.py            # writes oracle/libnbref.so

The oracle is compiled with -O2 -ffp-contract=off and no fast-math so that
every floating-point expression is evaluated as written.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "libnbref.so")
SRC = [os.path.join(HERE, "nbref.c")]
HDR = [os.path.join(HERE, "nbref.h")]


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in SRC + HDR)


def build(force: bool = False) -> str:
    if force or needs_build():
        tmp = LIB + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-Wall", "-Wextra", "-Wno-unused-parameter",
               "-o", tmp] + SRC + ["-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
