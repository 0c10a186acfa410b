"""Compile the plain-C FP64 oracle (``orc.c``, ``orc_moments.c``) into ``oracle/_build/liborc.so``.

Test infrastructure only: the product path never loads this library.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "orc.c"), os.path.join(HERE, "orc_moments.c")]
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liborc.so")


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and all(os.path.getmtime(LIB) >= os.path.getmtime(s) for s in SRCS)):
        return LIB
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=gnu11", "-fno-fast-math"]
    tmp = LIB + ".tmp%d" % os.getpid()
    try:
        subprocess.run(base + ["-fopenmp"] + SRCS + ["-o", tmp, "-lm"], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        # no OpenMP runtime: the oracle is still correct, just single-threaded
        subprocess.run(base + SRCS + ["-o", tmp, "-lm"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
