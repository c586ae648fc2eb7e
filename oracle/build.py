"""Compile the FP64 CPU oracle into oracle/liboracle_ba.so (test infrastructure)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, f) for f in ("ba_oracle.c", "gp_oracle.c")]
HDRS = [os.path.join(HERE, f) for f in ("ba_oracle.h", "gp_oracle.h")]
LIB = os.path.join(HERE, "liboracle_ba.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
            os.path.getmtime(f) for f in SRCS + HDRS):
        return LIB
    # -ffp-contract=off: every product and sum is rounded as written.
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-Wall", "-o", LIB + ".tmp", *SRCS, "-lm"]
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
