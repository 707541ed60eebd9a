"""Helpers for comparing a CUDA-built tree (exported blob) with the oracle.

Only test code: the Morton de-interleave and the per-node polynomial
evaluation below are written independently of both the CUDA library and the
oracle.
"""
from __future__ import annotations

import math

import numpy as np


def spread3(v):
    v = np.asarray(v, dtype=np.uint64) & np.uint64(0x1FFFFF)
    out = np.zeros_like(v)
    for b in range(21):
        out |= ((v >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b)
    return out


def compact3(c):
    c = np.asarray(c, dtype=np.uint64)
    out = np.zeros_like(c)
    for b in range(21):
        out |= ((c >> np.uint64(3 * b)) & np.uint64(1)) << np.uint64(b)
    return out


def quantise_np(x, lo, side):
    S = 2097152.0 / side
    t = (np.asarray(x, np.float64) - lo) * S
    q = np.floor(np.where(t >= 0, t, 0.0))
    q = np.where(t >= 2097152.0, 2097151.0, q)
    return q.astype(np.uint64)


def morton_np(x, y, z, lo=(0.0, 0.0, 0.0), side=1.0):
    return spread3(quantise_np(x, lo[0], side)) | (spread3(quantise_np(y, lo[1], side)) << np.uint64(1)) | \
        (spread3(quantise_np(z, lo[2], side)) << np.uint64(2))


def gpu_keys(ex, problem=0):
    """{(depth, ix, iy, iz): index} of one problem of an exported tree."""
    keys = {}
    mp = ex.morton_prefix()
    for i in range(ex.prefix.shape[0]):
        if int(ex.problem[i]) != problem:
            continue
        p = np.uint64(mp[i])
        keys[(int(ex.depth[i]), int(compact3(p)), int(compact3(p >> np.uint64(1))), int(compact3(p >> np.uint64(2))))] = i
    return keys


def oracle_keys(T):
    return {(int(T.depth[i]),) + tuple(int(a) for a in T.ixyz[i]): i for i in range(T.n_nodes)}


def exponents(p):
    return [(l, m, n) for l in range(p + 1) for m in range(p - l + 1) for n in range(p - l - m + 1)]


def node_poly(coef, p, key, lo, side, pts):
    """Value of a node polynomial (coefficients F in Alg. 2 order) at global points."""
    d, ix, iy, iz = key
    h = side / 2 ** (d + 1)
    c = [lo[0] + (2 * ix + 1) * h, lo[1] + (2 * iy + 1) * h, lo[2] + (2 * iz + 1) * h]
    u, v, w = ((pts[:, a] - c[a]) / h for a in range(3))
    val = np.zeros(pts.shape[0])
    for k, (l, m, n) in enumerate(exponents(p)):
        val += coef[k] * u ** l * v ** m * w ** n / (math.factorial(l) * math.factorial(m) * math.factorial(n))
    return val


def excluded_subtrees(T, ex, problem=0):
    """Keys below a decision flagged near tau on either side (excluded from the
    node-set comparison), plus the flagged nodes themselves."""
    bad = set()
    ok = oracle_keys(T)
    for k, i in ok.items():
        for o in range(8):
            if T.near_mask[i] & (1 << o):
                bad.add((k[0] + 1, 2 * k[1] + (o & 1), 2 * k[2] + ((o >> 1) & 1), 2 * k[3] + ((o >> 2) & 1)))
    gk = gpu_keys(ex, problem)
    for k, i in gk.items():
        for o in range(8):
            if ex.near_mask[i] & (1 << o):
                bad.add((k[0] + 1, 2 * k[1] + (o & 1), 2 * k[2] + ((o >> 1) & 1), 2 * k[3] + ((o >> 2) & 1)))

    def under(key):
        d, x, y, z = key
        while d > 0:
            if (d, x, y, z) in bad:
                return True
            d, x, y, z = d - 1, x >> 1, y >> 1, z >> 1
        return False
    return under


def compare_trees(T, ex, tol, n_poly_pts=6, seed=0, problem=0, data_xyz=None):
    """Assert that the exported CUDA tree matches the oracle tree T.

    Structure (node set, point counts, octant counts, degrees) must be
    bit-exact outside subtrees below near-tau decisions; node polynomials
    must agree within tol (absolute).  With data_xyz = (x, y, z) (the whole
    input, input order) the polynomials are compared at up to n_poly_pts of
    each node's own points -- where a least-squares fit is determined even
    when the node basis is ill conditioned; otherwise at random points of
    the node box."""
    under = excluded_subtrees(T, ex, problem)
    ok, gk = oracle_keys(T), gpu_keys(ex, problem)
    so = {k for k in ok if not under(k)}
    sg = {k for k in gk if not under(k)}
    assert so == sg, "node sets differ: only oracle %s, only gpu %s" % (sorted(so - sg)[:5], sorted(sg - so)[:5])
    rng = np.random.default_rng(seed)
    p = T.degree
    worst = 0.0
    for k in so:
        i, j = ok[k], gk[k]
        assert T.npts[i] == ex.count[j], k
        assert T.deg_used[i] == ex.deg_used[j], k
        assert np.array_equal(T.child_n[i], ex.child_n[j]), k
        assert (T.flags[i] & 4) == (ex.flags[j] & 4), k
        assert np.max(np.abs(T.child_E[i] - ex.child_E[j])) <= tol, k
        d = k[0]
        h = T.side / 2 ** d
        if data_xyz is not None:
            sel = ex.perm[ex.start[j] + rng.choice(int(ex.count[j]), min(n_poly_pts, int(ex.count[j])), replace=False)]
            pts = np.stack([data_xyz[0][sel], data_xyz[1][sel], data_xyz[2][sel]], axis=1)
        else:
            lo = np.array([T.lo[0] + k[1] * h, T.lo[1] + k[2] * h, T.lo[2] + k[3] * h])
            pts = lo + h * rng.uniform(0, 1, (n_poly_pts, 3))
        a = node_poly(T.coef[i], p, k, T.lo, T.side, pts)
        b = node_poly(ex.coef[j], p, k, T.lo, T.side, pts)
        worst = max(worst, float(np.max(np.abs(a - b))))
    assert worst <= tol, "node polynomial mismatch %g > %g" % (worst, tol)
    return worst
