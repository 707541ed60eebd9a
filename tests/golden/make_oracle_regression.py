"""Writes oracle_regression_small.txt: the oracle's tree on the small workload
(4096 uniform points, Franke values, p = 4, depth 3, min_pts 64, tol 1e-4).

Calls only oracle/ and the seeded input generators.  The file is a regression
record, not a correctness pin (the pins are in tests/test_oracle_pins.py): any
change to the oracle's arithmetic changes it, and the commit that rewrites it
must name the passage of the paper, or the reading of it, that justifies the
change.  Node table as text; coefficients and residual as SHA-256 digests of
their little-endian float64 bytes (the oracle uses only correctly rounded
operations in a fixed order, so the bytes are reproducible).

    python tests/golden/make_oracle_regression.py
"""
import hashlib
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import oracle as O  # noqa: E402
from paper_1511_01353_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "oracle_regression_small.txt")


def record():
    w = W.small()
    T = O.fit(w.x, w.y, w.z, w.f, w.degree, w.max_depth, w.min_pts, w.tol_rel)
    vals, _ = T.evaluate(w.xq, w.yq, w.zq)
    lines = ["# oracle tree of the small workload: %d points, p = %d, depth %d, min_pts %d, tol_rel %g"
             % (w.n, w.degree, w.max_depth, w.min_pts, w.tol_rel),
             "# written by tests/golden/make_oracle_regression.py (calls only oracle/)",
             "tau %s" % float(T.tau).hex(),
             "nodes %d" % T.n_nodes,
             "# depth ix iy iz npts flags deg_used refine_mask near_mask"]
    for i in range(T.n_nodes):
        lines.append("%d %d %d %d %d %d %d %d %d" % (T.depth[i], T.ixyz[i, 0], T.ixyz[i, 1], T.ixyz[i, 2],
                                                      T.npts[i], T.flags[i], T.deg_used[i], T.refine_mask[i],
                                                      T.near_mask[i]))
    for name, arr in (("coef", T.coef), ("resid", T.resid), ("eval", vals)):
        lines.append("sha256 %s %s" % (name, hashlib.sha256(np.ascontiguousarray(arr, "<f8").tobytes()).hexdigest()))
    return "\n".join(lines) + "\n"


if __name__ == "__main__":
    with open(OUT, "w") as fh:
        fh.write(record())
    print(OUT)
