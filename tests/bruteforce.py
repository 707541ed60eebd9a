"""Independent brute-force restatement of the free-mesh transform, used only
to pin the oracle on tiny inputs.

It shares nothing with oracle/: the basis comes from a lexicographic sort of
all exponent triples, octants from geometric comparisons against dyadic box
centres, and the least-squares fit from numpy's SVD solver (LAPACK gelsd)
instead of Householder QR.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def exponents(p):
    return sorted(t for t in itertools.product(range(p + 1), repeat=3) if sum(t) <= p)


def basis(p, u, v, w):
    E = exponents(p)
    cols = [u ** l * v ** m * w ** n / (math.factorial(l) * math.factorial(m) * math.factorial(n))
            for (l, m, n) in E]
    return np.stack(cols, axis=1)


def fmt_tree(x, y, z, f, p, max_depth, min_pts, tol_rel, lo=(0.0, 0.0, 0.0), side=1.0):
    """Returns {(depth, ix, iy, iz): dict(n, coef, childE)} and the final residual."""
    L = len(exponents(p))
    tau = tol_rel * float(np.max(np.abs(f)))
    r = np.array(f, dtype=np.float64)
    nodes = {}

    def visit(depth, ijk, idx):
        h = side / 2 ** (depth + 1)
        c = [lo[a] + (2 * ijk[a] + 1) * h for a in range(3)]
        u = (x[idx] - c[0]) / h
        v = (y[idx] - c[1]) / h
        w = (z[idx] - c[2]) / h
        A = basis(p, u, v, w)
        F, *_ = np.linalg.lstsq(A, r[idx], rcond=None)
        r[idx] = r[idx] - A @ F
        # children: geometric test against the box centre (upper half if >= centre)
        bx = (x[idx] >= c[0]).astype(int)
        by = (y[idx] >= c[1]).astype(int)
        bz = (z[idx] >= c[2]).astype(int)
        o = bx | (by << 1) | (bz << 2)
        childE = np.zeros(8)
        kids = []
        for oc in range(8):
            sel = idx[o == oc]
            if sel.size == 0:
                continue
            childE[oc] = math.sqrt(float(np.sum(r[sel] ** 2)) / sel.size)
            if depth + 1 <= max_depth and sel.size >= max(L, min_pts) and childE[oc] > tau:
                kids.append((oc, sel))
        nodes[(depth,) + tuple(ijk)] = dict(n=idx.size, coef=F, childE=childE)
        for oc, sel in kids:
            visit(depth + 1, (2 * ijk[0] + (oc & 1), 2 * ijk[1] + ((oc >> 1) & 1), 2 * ijk[2] + ((oc >> 2) & 1)), sel)

    visit(0, (0, 0, 0), np.arange(len(x)))
    return nodes, r, tau
