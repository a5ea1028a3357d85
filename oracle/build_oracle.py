"""Build the oracle's one C routine (order-exact pivot loop) in place.

TEST INFRASTRUCTURE.  ``python oracle/build_oracle.py`` writes
``oracle/_pivots.so``; the oracle's Python wrapper builds it on first use.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pivots.c")
OUT = os.path.join(HERE, "_pivots.so")


def build(force: bool = False) -> str:
    """Compile the order-exact pivot routine (Alg. 1) with gcc, with FMA
    contraction and fast math off so that every product and sum is the
    correctly rounded operation the source writes (OpenMP splits loops over
    grid points only); returns the library path."""
    if not force and os.path.exists(OUT) and os.path.getmtime(OUT) >= os.path.getmtime(SRC):
        return OUT
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-o", OUT + ".tmp", SRC, "-lm"]
    # use the hardware fused multiply-add when the host has one (the result
    # of fma() is the same correctly rounded value either way)
    try:
        flags = open("/proc/cpuinfo").read()
        if " fma " in flags and " avx2 " in flags:
            cmd[1:1] = ["-mfma", "-mavx2"]
    except OSError:
        pass
    subprocess.check_call(cmd)
    os.replace(OUT + ".tmp", OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
