"""Compile the FP64 CPU oracle (test infrastructure) into oracle/liboracle_vlb.so.

Plain gcc, -O2 with floating-point contraction off so every product and sum
rounds as written, and OpenMP for the loop over the cells of a step (each
cell's arithmetic is the same on any number of threads). Host-portable: no
-march flags, builds the same on x86-64 and aarch64.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle_vlb.so")
SRC = os.path.join(HERE, "vlb_oracle.c")
HDR = os.path.join(HERE, "vlb_oracle.h")


def _cc(out, src):
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-Wall", "-fPIC", "-shared", "-fopenmp",
           "-I", HERE, "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)


def build_oracle_copy(source_text: str, out_dir: str) -> str:
    """Compile a modified copy of the oracle source (tests that plant a
    mistake in the oracle) into out_dir; returns the library path."""
    src = os.path.join(out_dir, "vlb_oracle_copy.c")
    with open(src, "w") as fh:
        fh.write(source_text)
    out = os.path.join(out_dir, "liboracle_copy.so")
    _cc(out, src)
    return out


def build_oracle(force: bool = False) -> str:
    """Build the oracle library if it is missing or older than its sources."""
    if not force and os.path.exists(LIB):
        lt = os.path.getmtime(LIB)
        if lt >= os.path.getmtime(SRC) and lt >= os.path.getmtime(HDR):
            return LIB
    _cc(LIB, SRC)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
