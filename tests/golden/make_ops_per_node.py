"""Writes ops_per_node.txt: the algorithmic work of one evaluation of the local operator F per node
(Secs. 4.2-4.3 with the recompute rule of Sec. 2), counted by the FP64 oracle on converged fields of the
benchmark's workloads.

Every floating-point add, subtract, multiply, divide, square root, absolute value, comparison and libm call
that the oracle's evaluation of F executes counts 1 (the count is defined in oracle/alifmm_oracle.c).  The
benchmark divides (this count x nodes) by the sweep kernel's time to get its achieved rate.

Run: python tests/golden/make_ops_per_node.py   (calls only oracle/ and the seeded input generators)
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_2302_10988_gb300 import workloads as W  # noqa: E402

# the fields counted: (workload, sample, source)
FIELDS = {
    "weld_batch": [(b, s) for b in (0, 3, 7, 12, 21, 30, 44, 61) for s in (0, 17)],
    "weld_single": [(0, s) for s in (0, 9, 16, 27)],
}


def count(wl, b, s):
    smp = wl.samples[b]
    mats = [O.mat_from_voigt(c6, rho) for c6, rho in wl.materials]
    M = O.OMedium.from_regions(smp.nx, smp.ny, smp.h, smp.region_map, smp.region_theta, wl.region_material, mats)
    fr, t0 = O.init_radius(M, *smp.src[s], 2)
    tau = O.fmm(M, fr, t0)[0]
    return O.ops_of_F_all(M, fr, tau)


def workload(name):
    return W.weld_batch() if name == "weld_batch" else W.weld_single()


def main():
    lines = ["# workload sample source ops nodes  (one evaluation of F at every non-frozen node, oracle count)"]
    for name, fields in FIELDS.items():
        wl = workload(name)
        tot_ops = tot_n = 0
        for b, s in fields:
            ops, n = count(wl, b, s)
            lines.append(f"{name} {b} {s} {ops} {n}")
            tot_ops += ops
            tot_n += n
        lines.append(f"# {name}: {tot_ops / tot_n:.2f} operations per node")
    with open(os.path.join(HERE, "ops_per_node.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


def read(path=os.path.join(HERE, "ops_per_node.txt")):
    """{workload: operations per node} from the stored file."""
    acc = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        name, b, s, ops, n = line.split()
        o, m = acc.get(name, (0, 0))
        acc[name] = (o + int(ops), m + int(n))
    return {k: o / m for k, (o, m) in acc.items()}


if __name__ == "__main__":
    main()
