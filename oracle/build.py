"""Build the plain-C FP64 oracle into ``oracle/_build/liboracle.so``.

Test infrastructure only: the oracle is a checker.  ``-ffp-contract=off``
keeps gcc from fusing multiply-adds, so x86 and aarch64 builds round alike.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "swpic_oracle.c"), os.path.join(HERE, "swpic2d_oracle.c")]
OUT_DIR = os.path.join(HERE, "_build")
OUT = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(OUT)
            and all(os.path.getmtime(OUT) >= os.path.getmtime(s) for s in SRCS)):
        return OUT
    tmp = OUT + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-std=c99", "-Wall", "-fPIC", "-shared",
            "-ffp-contract=off", "-fno-fast-math", "-o", tmp, *SRCS, "-lm"]
    # OpenMP only serves or_set_threads (timing on all host cores); without it
    # the oracle builds serial and or_set_threads reports 1 thread
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(base, check=True)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
