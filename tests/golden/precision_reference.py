"""Oracle fields for the storage-precision comparison.

Runs the FP64 CPU oracle (and nothing else) on the 64^3 channel instance of
workloads.precision_instance and writes rho, u and the conservation totals
after each checkpoint to precision64_oracle.npz beside this file (about 8 MB
per checkpoint, not committed). `bench.py --workload precision` compares the
GPU's 16-bit, FP32 and FP64 runs of the same instance with these fields.

The oracle advances a 64^3 D3Q19 mesh at a few hundredths of a million cell
updates per second on one core, so 1000 steps take one to two hours.

usage: python -m tests.golden.precision_reference [--n 64] [--steps 200,1000]
"""
import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import OracleSim  # noqa: E402
from paper_2401_17183_gb300 import workloads as W  # noqa: E402


def out_path(n):
    return os.path.join(HERE, "precision%d_oracle.npz" % n)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--steps", default="200,1000")
    a = ap.parse_args()
    marks = sorted(int(s) for s in a.steps.split(","))
    mesh, prm, rho, u = W.precision_instance(a.n)
    o = OracleSim(mesh, prm)
    o.init(rho, u)
    out = {"n": a.n, "steps": np.array(marks)}
    mass0 = o.moments()["mass"]
    out["mass0"] = mass0
    t0, done = time.time(), 0
    for k in marks:
        o.step(k - done)
        done = k
        mo = o.moments()
        out["rho_%d" % k] = mo["rho"]
        out["u_%d" % k] = mo["u"]
        out["mass_%d" % k] = mo["mass"]
        np.savez(out_path(a.n), **out)
        print("step %d: %.0f s, mass drift %.3e" % (k, time.time() - t0, mo["mass"] / mass0 - 1.0), flush=True)


if __name__ == "__main__":
    main()
