"""Build the CPU oracle (test infrastructure only) into oracle/_build/.

Plain gcc, FP64, no FMA contraction (so the oracle's rounding is the C
source's own), OpenMP over elements for the CPU-baseline timing.  Host code
only: builds unchanged on x86_64 and aarch64 (no -march flags).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "dg_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libdg_oracle.so")


def build_oracle(force=False, extra_flags=(), out=None):
    """Compile dg_oracle.c; returns the path of the shared library.

    `extra_flags` lets a test compile a variant (e.g. with a planted mistake
    selected by a -D flag) into a separate file given by `out`.
    """
    out = out or LIB
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-std=c11", "-Wall", *extra_flags,
           "-o", out + ".tmp", SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


if __name__ == "__main__":
    print(build_oracle(force="--force" in sys.argv))
