"""Compile the FP64 CPU oracle (test infrastructure) into oracle/liboracle_vlb.so.

Plain gcc, -O2 with floating-point contraction off so every product and sum
rounds as written. Host-portable: no -march flags, builds the same on x86-64
and aarch64.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle_vlb.so")
SRC = os.path.join(HERE, "vlb_oracle.c")
HDR = os.path.join(HERE, "vlb_oracle.h")


def build_oracle(force: bool = False) -> str:
    """Build the oracle library if it is missing or older than its sources."""
    if not force and os.path.exists(LIB):
        lt = os.path.getmtime(LIB)
        if lt >= os.path.getmtime(SRC) and lt >= os.path.getmtime(HDR):
            return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-Wall", "-fPIC", "-shared",
           "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
