"""ctypes binding of the plain FP64 C oracle (oracle/fmt_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()``
and the CPU legs of bench.py (cpu_baseline, --impl reference), never by the
product path.

The oracle follows Alg. 1 (recursive octree decomposition of the residual)
and Alg. 2 (geometric-moment Vandermonde, Householder QR, F = R^-1 Q^T f,
f <- f - Lambda F) of Challacombe, arXiv 1511.01353, and evaluates the tree
interpolant as the sum over a target's octree path of Lambda(r) . F
(Sec. 2, end).  Parity pins: tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmt_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

FLAG_NEAR_TAU = 1
FLAG_RANK = 2
FLAG_DEG_CLAMPED = 4


def compile_library(src: str, out: str, extra=()) -> None:
    """gcc build of an oracle source: IEEE FP64, no contraction, OpenMP;
    extra flags are appended (the sanitizer test adds ASan/UBSan)."""
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", *extra, "-o", out, src, "-lm"]
    subprocess.run(cmd, check=True)


def build(force: bool = False) -> str:
    """Compile oracle/fmt_oracle.c into oracle/liboracle.so when it is stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        compile_library(_SRC, tmp)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    """The loaded oracle library.  FMT_ORACLE_LIB names another build of an
    oracle source to load instead (the mutation test loads deliberately broken
    copies this way, in child processes)."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("FMT_ORACLE_LIB") or build()
            L = ctypes.CDLL(path)
            d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
            P = ctypes.c_void_p
            L.ora_nmono.argtypes = [i32]
            L.ora_nmono.restype = i32
            L.ora_monomials.argtypes = [i32, d, d, d, P]
            L.ora_monomials.restype = None
            L.ora_quantise.argtypes = [d, d, d]
            L.ora_quantise.restype = ctypes.c_uint32
            L.ora_fit_node.argtypes = [i32, i64, P, P, P, P, P]
            L.ora_fit_node.restype = i32
            L.ora_fit.argtypes = [i32, i32, i32, d, P, d, i64, P, P, P, P, i32, ctypes.POINTER(P)]
            L.ora_fit.restype = i32
            L.ora_num_nodes.argtypes = [P]
            L.ora_num_nodes.restype = i64
            L.ora_tau.argtypes = [P]
            L.ora_tau.restype = d
            L.ora_maxabs.argtypes = [P]
            L.ora_maxabs.restype = d
            L.ora_get_nodes.argtypes = [P] * 13
            L.ora_get_nodes.restype = None
            L.ora_get_residual.argtypes = [P, P]
            L.ora_get_residual.restype = None
            L.ora_eval.argtypes = [P, i64, P, P, P, P, P]
            L.ora_eval.restype = i32
            L.ora_free.argtypes = [P]
            L.ora_free.restype = None
            L.ora_num_threads.argtypes = []
            L.ora_num_threads.restype = i32
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def nmono(p: int) -> int:
    return int(lib().ora_nmono(p))


def monomials(p: int, u: float, v: float, w: float) -> np.ndarray:
    out = np.zeros(nmono(p), dtype=np.float64)
    lib().ora_monomials(p, u, v, w, _ptr(out))
    return out


def quantise(lo: float, side: float, x: float) -> int:
    return int(lib().ora_quantise(lo, side, x))


def fit_node(q: int, u, v, w, r):
    """Alg. 2 on points already in a node frame: returns (F, r_new, flags)."""
    u, v, w = _f64(u), _f64(v), _f64(w)
    r2 = _f64(r).copy()
    F = np.zeros(nmono(q), dtype=np.float64)
    fl = lib().ora_fit_node(q, u.shape[0], _ptr(u), _ptr(v), _ptr(w), _ptr(r2), _ptr(F))
    if fl < 0:
        raise MemoryError("oracle fit_node failed")
    return F, r2, int(fl)


@dataclasses.dataclass
class OracleTree:
    degree: int
    nmono: int
    max_depth: int
    min_pts: int
    tol_rel: float
    tau: float
    maxabs: float
    lo: tuple
    side: float
    depth: np.ndarray      # [K] int32
    ixyz: np.ndarray       # [K,3] uint32 box coordinates at the node's depth
    npts: np.ndarray       # [K] int64
    flags: np.ndarray      # [K] int32
    deg_used: np.ndarray   # [K] int32
    parent: np.ndarray     # [K] int64
    child: np.ndarray      # [K,8] int64 (-1 = absent)
    child_E: np.ndarray    # [K,8] RMS residual of each octant after this node's fit
    child_n: np.ndarray    # [K,8] points per octant
    near_mask: np.ndarray  # [K] uint32
    refine_mask: np.ndarray  # [K] uint32
    coef: np.ndarray       # [K, nmono] F in Alg. 2 order
    resid: np.ndarray      # [N] final residual in input order
    _handle: object = None

    def __del__(self):
        h = self._handle
        if h is not None and _lib is not None:
            _lib.ora_free(h)
            self._handle = None

    @property
    def n_nodes(self):
        return int(self.depth.shape[0])

    def evaluate(self, xq, yq, zq):
        xq, yq, zq = _f64(xq), _f64(yq), _f64(zq)
        out = np.zeros(xq.shape[0], dtype=np.float64)
        nout = ctypes.c_int64(0)
        rc = lib().ora_eval(self._handle, xq.shape[0], _ptr(xq), _ptr(yq), _ptr(zq), _ptr(out),
                            ctypes.cast(ctypes.byref(nout), ctypes.c_void_p))
        if rc:
            raise RuntimeError("oracle eval failed: %d" % rc)
        return out, int(nout.value)


def fit(x, y, z, f, degree, max_depth, min_pts, tol_rel, lo=(0.0, 0.0, 0.0), side=1.0, mode="dfs"):
    """Alg. 1 over the whole point set.  mode: 'dfs' (serial, as printed),
    'omp' (depth-first with OpenMP tasks; identical results), 'bfs'."""
    x, y, z, f = _f64(x), _f64(y), _f64(z), _f64(f)
    lo_a = np.asarray(lo, dtype=np.float64)
    h = ctypes.c_void_p()
    m = {"dfs": 0, "omp": 1, "bfs": 2}[mode]
    rc = lib().ora_fit(degree, max_depth, min_pts, tol_rel, _ptr(lo_a), side, x.shape[0], _ptr(x), _ptr(y),
                       _ptr(z), _ptr(f), m, ctypes.byref(h))
    if rc == 1:
        raise ValueError("oracle: invalid arguments")
    if rc:
        raise MemoryError("oracle: out of memory")
    L = lib()
    K = int(L.ora_num_nodes(h))
    nm = nmono(degree)
    depth = np.zeros(K, np.int32)
    ixyz = np.zeros((K, 3), np.uint32)
    npts = np.zeros(K, np.int64)
    flags = np.zeros(K, np.int32)
    deg_used = np.zeros(K, np.int32)
    parent = np.zeros(K, np.int64)
    child = np.zeros((K, 8), np.int64)
    child_E = np.zeros((K, 8), np.float64)
    child_n = np.zeros((K, 8), np.int64)
    near = np.zeros(K, np.uint32)
    ref = np.zeros(K, np.uint32)
    coef = np.zeros((K, nm), np.float64)
    L.ora_get_nodes(h, _ptr(depth), _ptr(ixyz), _ptr(npts), _ptr(flags), _ptr(deg_used), _ptr(parent),
                    _ptr(child), _ptr(child_E), _ptr(child_n), _ptr(near), _ptr(ref), _ptr(coef))
    resid = np.zeros(x.shape[0], np.float64)
    L.ora_get_residual(h, _ptr(resid))
    return OracleTree(degree, nm, max_depth, min_pts, tol_rel, float(L.ora_tau(h)), float(L.ora_maxabs(h)),
                      tuple(float(a) for a in lo), float(side), depth, ixyz, npts, flags, deg_used, parent, child,
                      child_E, child_n, near, ref, coef, resid, h)


def num_threads() -> int:
    return int(lib().ora_num_threads())
