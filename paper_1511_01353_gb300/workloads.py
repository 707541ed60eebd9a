"""Seeded synthetic workloads for the free-mesh transform (FMT).

This module only draws inputs: point clouds, sample values of the test
functions and target points.  It holds none of the method's arithmetic
(no quantisation, no basis, no fit), so both the CPU oracle and the CUDA
path may take their inputs from here.

Random numbers come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11), written out below
from its published definition so that every machine draws identical bits.

Workloads follow the paper's experiments (random grids in [0,1]^3 with
3-D Franke values, Sec. 3 Eq. eqF1 and Sec. 4) at the sizes of the
benchmark configurations:

* ``small``  : 4096 uniform points, p=4, depth 3, min 64, tol 1e-4, 1e4 targets
* ``scale``  : 1e6 points (half uniform, half in 8 Gaussian clusters,
               sigma 0.05, centres U[0.2,0.8]^3, rejection into [0,1)^3),
               p=8, depth 7, min 128, tol 1e-8, 1e7 targets
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 1511013530

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds.

    ctr: four uint32 arrays (broadcastable), key: two uint32 scalars.
    Returns four uint32 arrays.  Each round multiplies words 0 and 2 by
    the Philox constants, swaps hi/lo halves and xors in the round key;
    the key is bumped by the Weyl constants between rounds.
    """
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _MASK for c in ctr)
    k0 = np.uint64(int(key[0]) & 0xFFFFFFFF)
    k1 = np.uint64(int(key[1]) & 0xFFFFFFFF)
    for _ in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + _W0) & _MASK
        k1 = (k1 + _W1) & _MASK
    return tuple(c.astype(np.uint32) for c in (c0, c1, c2, c3))


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0,1) from counters (i, stream, 0, 0), i = offset/2 ...

    Each counter yields two doubles with 53 random bits each
    (27 high bits from one word, 26 from the next).  ``offset`` must be even.
    """
    if n <= 0:
        return np.zeros(0, dtype=np.float64)
    assert offset % 2 == 0
    ncounter = (n + 1) // 2
    i = np.arange(offset // 2, offset // 2 + ncounter, dtype=np.uint64)
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    z = np.zeros_like(i)
    w0, w1, w2, w3 = philox4x32_10((i, np.full_like(i, stream), z, z), key)
    a = np.empty(2 * ncounter, dtype=np.float64)
    a[0::2] = ((w0 >> 5).astype(np.float64) * 67108864.0 + (w1 >> 6).astype(np.float64))
    a[1::2] = ((w2 >> 5).astype(np.float64) * 67108864.0 + (w3 >> 6).astype(np.float64))
    a *= 2.0 ** -53
    return a[:n]


def normal(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n standard normals by Box-Muller on consecutive uniform pairs.

    Normal 2s uses cos, 2s+1 uses sin of the pair (u[2s], u[2s+1]) drawn at
    uniform offset ``offset + 2s``; 1-u keeps the logarithm finite.
    """
    if n <= 0:
        return np.zeros(0, dtype=np.float64)
    npair = (n + 1) // 2
    u = uniform(seed, stream, 2 * npair, offset)
    rad = np.sqrt(-2.0 * np.log1p(-u[0::2]))
    ang = 2.0 * math.pi * u[1::2]
    z = np.empty(2 * npair, dtype=np.float64)
    z[0::2] = rad * np.cos(ang)
    z[1::2] = rad * np.sin(ang)
    return z[:n]


def franke_bj(x, y, z):
    """3-D Franke function as written in the benchmark configurations:
    the second exponential has (9y+1)/10 and (9z+1)/10 unsquared."""
    x, y, z = (np.asarray(a, dtype=np.float64) for a in (x, y, z))
    return (0.75 * np.exp(-((9 * x - 2) ** 2 + (9 * y - 2) ** 2 + (9 * z - 2) ** 2) / 4)
            + 0.75 * np.exp(-(9 * x + 1) ** 2 / 49 - (9 * y + 1) / 10 - (9 * z + 1) / 10)
            + 0.5 * np.exp(-((9 * x - 7) ** 2 + (9 * y - 3) ** 2 + (9 * z - 5) ** 2) / 4)
            - 0.2 * np.exp(-(9 * x - 4) ** 2 - (9 * y - 7) ** 2 - (9 * z - 5) ** 2))


def franke_paper(x, y, z):
    """3-D Franke function of Sec. 3, Eq. eqF1 (second term squares 9y+1, 9z+1)."""
    x, y, z = (np.asarray(a, dtype=np.float64) for a in (x, y, z))
    return (0.75 * (np.exp(-0.25 * ((9 * x - 2) ** 2 + (9 * y - 2) ** 2 + (9 * z - 2) ** 2))
                    + np.exp(-(9 * x + 1) ** 2 / 49 - (9 * y + 1) ** 2 / 10 - (9 * z + 1) ** 2 / 10))
            + 0.5 * np.exp(-0.25 * ((9 * x - 7) ** 2 + (9 * y - 3) ** 2 + (9 * z - 5) ** 2))
            - 0.2 * np.exp(-(9 * x - 4) ** 2 - (9 * y - 7) ** 2 - (9 * z - 5) ** 2))


def uniform_points(seed: int, stream: int, n: int):
    a = uniform(seed, stream, 3 * n).reshape(n, 3) if n > 0 else np.zeros((0, 3))
    return np.ascontiguousarray(a[:, 0]), np.ascontiguousarray(a[:, 1]), np.ascontiguousarray(a[:, 2])


def clustered_points(seed: int, stream: int, n: int, centre, sigma: float):
    """n points from an isotropic Gaussian around ``centre``; candidates that
    fall outside [0,1)^3 are rejected and the next candidate is taken.
    Candidate t uses normals 3t, 3t+1, 3t+2 of the stream, so the result
    does not depend on how candidates are batched."""
    out = np.zeros((0, 3))
    t0 = 0                                   # first candidate of the batch (kept even)
    batch = max(64, 2 * n + (n % 2))         # even, so normal 3*t0 starts a Box-Muller pair
    c = np.asarray(centre, dtype=np.float64).reshape(1, 3)
    while out.shape[0] < n:
        z = normal(seed, stream, 3 * batch, offset=3 * t0)
        cand = c + sigma * z.reshape(batch, 3)
        ok = np.all((cand >= 0.0) & (cand < 1.0), axis=1)
        out = np.concatenate([out, cand[ok]], axis=0)
        t0 += batch
    out = out[:n]
    return np.ascontiguousarray(out[:, 0]), np.ascontiguousarray(out[:, 1]), np.ascontiguousarray(out[:, 2])


@dataclasses.dataclass
class Workload:
    name: str
    degree: int
    max_depth: int
    min_pts: int
    tol_rel: float
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    f: np.ndarray
    xq: np.ndarray
    yq: np.ndarray
    zq: np.ndarray

    @property
    def n(self):
        return int(self.x.shape[0])

    @property
    def m(self):
        return int(self.xq.shape[0])


def small(n: int = 4096, n_targets: int = 10_000, seed: int = SEED_BASE + 0) -> Workload:
    """Uniform cloud with 3-D Franke values, p=4, depth 3, min 64, tol 1e-4."""
    x, y, z = uniform_points(seed, 1, n)
    xq, yq, zq = uniform_points(seed, 7, n_targets)
    return Workload("small_fp64_n%d_p4_d3" % n, 4, 3, 64, 1e-4, x, y, z, franke_bj(x, y, z), xq, yq, zq)


def scale(n: int = 1_000_000, n_targets: int = 10_000_000, seed: int = SEED_BASE + 1,
          degree: int = 8, max_depth: int = 7, min_pts: int = 128, tol_rel: float = 1e-8) -> Workload:
    """Half uniform, half in 8 Gaussian clusters (sigma 0.05, centres U[0.2,0.8]^3)."""
    n_uni = n // 2
    n_clu = n - n_uni
    xs, ys, zs = [], [], []
    x, y, z = uniform_points(seed, 1, n_uni)
    xs.append(x); ys.append(y); zs.append(z)
    centres = 0.2 + 0.6 * uniform(seed, 2, 24).reshape(8, 3)
    per = [n_clu // 8 + (1 if c < n_clu % 8 else 0) for c in range(8)]
    for c in range(8):
        x, y, z = clustered_points(seed, 100 + c, per[c], centres[c], 0.05)
        xs.append(x); ys.append(y); zs.append(z)
    x, y, z = np.concatenate(xs), np.concatenate(ys), np.concatenate(zs)
    xq, yq, zq = uniform_points(seed, 7, n_targets)
    return Workload("scale_fp64_n%d_p%d_d%d" % (n, degree, max_depth), degree, max_depth, min_pts, tol_rel,
                    x, y, z, franke_bj(x, y, z), xq, yq, zq)


def errors(pred, truth):
    """E_rms and E_inf of Sec. 4 (RMS and max absolute deviation)."""
    d = np.asarray(pred, dtype=np.float64) - np.asarray(truth, dtype=np.float64)
    if d.size == 0:
        return 0.0, 0.0
    return float(np.sqrt(np.mean(d * d))), float(np.max(np.abs(d)))


@dataclasses.dataclass
class Batch:
    """Many independent problems, concatenated (problem i owns offsets[i] ..
    offsets[i+1]-1 of the point arrays and toff[i] .. toff[i+1]-1 of the
    targets)."""
    name: str
    max_depth: int
    min_pts: int
    tol_rel: float
    offsets: np.ndarray
    degrees: np.ndarray
    boxes: np.ndarray        # [P, 4]: lo x, lo y, lo z, side
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    f: np.ndarray
    toff: np.ndarray
    xq: np.ndarray
    yq: np.ndarray
    zq: np.ndarray
    tprob: np.ndarray        # problem of every target (int32)
    fkind: list              # per problem: ("franke", shift, scale) or ("gauss", centres, exps, weights)
    cloud: list = dataclasses.field(default_factory=list)  # per problem: "uniform" or "clusters" 

    @property
    def n_problems(self):
        return int(self.offsets.shape[0] - 1)

    def truth(self, i, x, y, z):
        """The generating function of problem i at (x, y, z)."""
        return _batch_value(self.fkind[i], x, y, z)


def _batch_value(kind, x, y, z):
    if kind[0] == "franke":
        _, shift, scale = kind
        return franke_bj(0.5 + scale * (x - 0.5) + shift[0], 0.5 + scale * (y - 0.5) + shift[1],
                         0.5 + scale * (z - 0.5) + shift[2])
    _, cen, ex, wt = kind
    v = np.zeros_like(np.asarray(x, dtype=np.float64))
    for c, a, wk in zip(cen, ex, wt):
        v = v + wk * np.exp(-a * ((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2))
    return v


def batch(n_problems: int = 4096, n_min: int = 256, n_max: int = 65536, deg_min: int = 4, deg_max: int = 10,
          targets_per_problem: int = 1000, tol_rel: float = 1e-6, max_depth: int = 8, min_pts: int = 0,
          seed: int = SEED_BASE + 3) -> Batch:
    """Independent problems shaped like the batched configuration: point counts
    log-uniform in [n_min, n_max]; uniform clouds or 1-8 Gaussian clusters
    (sigma U[0.02, 0.2], centres U[0.2, 0.8]^3, rejected into [0,1)^3);
    degree uniform in [deg_min, deg_max]; values a shifted/scaled Franke
    function (shift U[-0.2,0.2]^3, scale U[0.5,2]) or a sum of 1-16 Gaussians
    (centres U[0,1]^3, exponent U[1,50], weight N(0,1)).  The targets of a
    problem are a fresh sample of the same cloud (uniform or the same
    clusters), so they lie where the problem has data."""
    P = n_problems
    u = uniform(seed, 1, 16 * P).reshape(P, 16)
    counts = np.floor(np.exp(np.log(n_min) + u[:, 0] * (np.log(n_max) - np.log(n_min)))).astype(np.int64)
    counts = np.clip(counts, n_min, n_max)
    degrees = (deg_min + np.floor(u[:, 1] * (deg_max - deg_min + 1))).astype(np.int32)
    degrees = np.minimum(degrees, deg_max)
    nt = targets_per_problem
    xs, ys, zs, fs, kinds, txs, tys, tzs, clouds = [], [], [], [], [], [], [], [], []
    for i in range(P):
        n = int(counts[i])
        if u[i, 2] < 0.5:
            x, y, z = uniform_points(seed, 1000 + i, n)
            tx, ty, tz = uniform_points(seed, 1000000 + i, nt)
            clouds.append("uniform")
        else:
            k = 1 + int(u[i, 3] * 8) if u[i, 3] < 1.0 else 8
            sig = 0.02 + 0.18 * u[i, 4]
            cen = 0.2 + 0.6 * uniform(seed, 200000 + i, 3 * k).reshape(k, 3)

            def cloud(cnt, base):
                per = [cnt // k + (1 if c < cnt % k else 0) for c in range(k)]
                parts = [clustered_points(seed, base + 8 * i + c, per[c], cen[c], sig)
                         for c in range(k) if per[c] > 0]
                return (np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts]),
                        np.concatenate([p[2] for p in parts]))
            x, y, z = cloud(n, 400000)
            tx, ty, tz = cloud(nt, 1200000)
            clouds.append("clusters")
        if u[i, 5] < 0.5:
            shift = -0.2 + 0.4 * u[i, 6:9]
            scale = 0.5 + 1.5 * u[i, 9]
            kind = ("franke", shift, scale)
        else:
            ng = 1 + int(u[i, 10] * 16) if u[i, 10] < 1.0 else 16
            gu = uniform(seed, 600000 + i, 4 * ng).reshape(ng, 4)
            kind = ("gauss", gu[:, :3], 1.0 + 49.0 * gu[:, 3], normal(seed, 800000 + i, ng))
        xs.append(x); ys.append(y); zs.append(z)
        txs.append(tx); tys.append(ty); tzs.append(tz)
        fs.append(_batch_value(kind, x, y, z))
        kinds.append(kind)
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    tprob = np.repeat(np.arange(P, dtype=np.int32), nt)
    boxes = np.tile(np.array([0.0, 0.0, 0.0, 1.0]), (P, 1))
    return Batch("batch_fp64_%dproblems_p%d-%d" % (P, deg_min, deg_max), max_depth, min_pts, tol_rel, offsets,
                 degrees, boxes, np.concatenate(xs), np.concatenate(ys), np.concatenate(zs), np.concatenate(fs),
                 np.arange(P + 1, dtype=np.int64) * nt, np.concatenate(txs), np.concatenate(tys),
                 np.concatenate(tzs), tprob, kinds, clouds)


@dataclasses.dataclass
class ServeRequest:
    arrival: float           # seconds after the start of the stream
    precision: str           # "fp64" or "mixed"
    degree: int
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    f: np.ndarray
    xq: np.ndarray
    yq: np.ndarray
    zq: np.ndarray


def serve_stream(n_requests: int = 48, rate: float = 200.0, n_min: int = 1000, n_max: int = 2_000_000,
                 t_min: int = 1, t_max: int = 1_000_000, deg_min: int = 4, deg_max: int = 10,
                 seed: int = SEED_BASE + 4) -> list:
    """Fit+evaluate requests shaped like the serving configuration: Poisson
    arrivals at `rate` per second; point counts log-uniform in [n_min,
    n_max], target counts log-uniform in [t_min, t_max]; degree uniform in
    [deg_min, deg_max]; clouds and values from the batched recipe's
    generators (uniform or 1-8 Gaussian clusters; shifted/scaled Franke or
    Gaussian sums), the targets a fresh sample of the same cloud; each
    request FP64 or mixed precision with probability 1/2."""
    R = n_requests
    u = uniform(seed, 1, 16 * R).reshape(R, 16)
    arrivals = np.cumsum(-np.log(1.0 - u[:, 0]) / rate)
    counts = np.floor(np.exp(np.log(n_min) + u[:, 1] * (np.log(n_max) - np.log(n_min)))).astype(np.int64)
    counts = np.clip(counts, n_min, n_max)
    tcounts = np.floor(np.exp(np.log(t_min) + u[:, 2] * (np.log(t_max) - np.log(t_min)))).astype(np.int64)
    tcounts = np.clip(tcounts, t_min, t_max)
    degrees = np.minimum(deg_min + np.floor(u[:, 3] * (deg_max - deg_min + 1)), deg_max).astype(np.int32)
    out = []
    for i in range(R):
        n, nt = int(counts[i]), int(tcounts[i])
        if u[i, 4] < 0.5:
            x, y, z = uniform_points(seed, 1000 + i, n)
            tx, ty, tz = uniform_points(seed, 1000000 + i, nt)
        else:
            k = 1 + int(u[i, 5] * 8) if u[i, 5] < 1.0 else 8
            sig = 0.02 + 0.18 * u[i, 6]
            cen = 0.2 + 0.6 * uniform(seed, 200000 + i, 3 * k).reshape(k, 3)

            def cloud(cnt, base):
                per = [cnt // k + (1 if c < cnt % k else 0) for c in range(k)]
                parts = [clustered_points(seed, base + 8 * i + c, per[c], cen[c], sig)
                         for c in range(k) if per[c] > 0]
                return (np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts]),
                        np.concatenate([p[2] for p in parts]))
            x, y, z = cloud(n, 400000)
            tx, ty, tz = cloud(nt, 1200000)
        if u[i, 7] < 0.5:
            kind = ("franke", -0.2 + 0.4 * u[i, 8:11], 0.5 + 1.5 * u[i, 11])
        else:
            ng = 1 + int(u[i, 12] * 16) if u[i, 12] < 1.0 else 16
            gu = uniform(seed, 600000 + i, 4 * ng).reshape(ng, 4)
            kind = ("gauss", gu[:, :3], 1.0 + 49.0 * gu[:, 3], normal(seed, 800000 + i, ng))
        out.append(ServeRequest(float(arrivals[i]), "mixed" if u[i, 13] < 0.5 else "fp64", int(degrees[i]),
                                x, y, z, _batch_value(kind, x, y, z), tx, ty, tz))
    return out
