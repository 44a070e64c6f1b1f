"""Write the golden fixtures of this folder from the FP64 oracle alone.

    python tests/golden/make_golden.py

visited_parallel64_linear.txt
    The visited (line, node) set of the 64 x 64 degree-1 parallel workload
    (90 angles a pi / 90, offsets -48 + b, b = 0..95): the number of nonzero
    pairs per view and in all, by brute force over every node (the open
    support |y~| < w of Sec. IV.A with w = (n + 1)(|cos| + |sin|) / 2).  The
    total, 938,120, was also found by an independent brute-force count.
footprint_values.txt
    phi_theta(y) of Prop. 1 (eq. xsa), degrees 0..3, at fixed angles and
    offsets, from the oracle's exact piecewise Gauss-Legendre convolution.
    The same values are pinned outside the oracle by the printed degree-1
    closed form (Sec. III.C), the Dirac case at theta = 0 and quadrature of
    the basis along the line (tests/test_oracle_footprint.py).
"""
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle      # noqa: E402
import workloads   # noqa: E402

ANGLES = [0.0, 0.1, 0.3, math.pi / 4, 1.0, 1.3, 2.0]
OFFSETS = [0.0, 0.25, 0.5, 0.9, 1.4, 1.9]


def visited_rows():
    wl = workloads.workload("parallel64_linear")
    geo = wl.geometry
    th, yy = oracle.lines_parallel(geo.view_angle.astype(np.float64), geo.n_det, geo.det0, geo.ddet)
    counts, _ = oracle.visited(oracle.Grid(wl.n, wl.n, wl.degree, wl.h), th, yy, brute=True)
    return counts.reshape(geo.view_angle.size, geo.n_det).sum(axis=1), int(counts.sum())


def footprint_rows():
    rows = []
    for n in range(4):
        for th in ANGLES:
            for y in OFFSETS:
                rows.append((n, th, y, oracle.footprint(n, th, y)))
    return rows


def main():
    oracle.build()
    per_view, total = visited_rows()
    with open(os.path.join(HERE, "visited_parallel64_linear.txt"), "w") as f:
        f.write("# nonzero (line, node) pairs of parallel64_linear (64 x 64, degree 1, 90 x 96 lines)\n")
        f.write("# written by tests/golden/make_golden.py from the FP64 oracle (brute force, Sec. IV.A)\n")
        f.write(f"total {total}\n")
        for v, c in enumerate(per_view):
            f.write(f"view {v} {int(c)}\n")
    with open(os.path.join(HERE, "footprint_values.txt"), "w") as f:
        f.write("# phi_theta(y) of Prop. 1 (eq. xsa): degree, theta, y, value\n")
        f.write("# written by tests/golden/make_golden.py from the FP64 oracle\n")
        for n, th, y, v in footprint_rows():
            f.write(f"{n} {th!r} {y!r} {v!r}\n")


if __name__ == "__main__":
    main()
