"""Thin ctypes binding of libfmt (include/fmt.h).

The functions keep the C names (oct_build, fit_level, refine, evaluate,
fmt_tree_stats, fmt_tree_export, fmt_tree_import, fmt_tree_free,
fmt_last_error, fmt_nmono) and only marshal arguments: device buffers are
torch CUDA tensors (float64, contiguous), streams are torch.cuda.Stream or
None (torch's current stream).  All arithmetic runs in the library's CUDA
kernels; there is no CPU fallback: loading fails loudly when libfmt.so is
missing or cannot be built.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfmt.so")

FMT_OK, FMT_EINVAL, FMT_ENOMEM, FMT_ECUDA, FMT_ETIMEOUT, FMT_EINTERNAL = range(6)
FMT_FP64, FMT_MIXED = 0, 1
FMT_FLAG_NEAR_TAU, FMT_FLAG_RANK, FMT_FLAG_DEG_CLAMPED, FMT_FLAG_MIXED = 1, 2, 4, 8
FMT_FLAG_MIXED_SLOW, FMT_FLAG_MIXED_PIVOT, FMT_FLAG_MIXED_FP64 = 16, 32, 64
MIXED_MAX_DEGREE = 9
MIXED_FP64_MAX_DEGREE = 10
MIXED_MAX_SWEEPS = 3
FMT_OPT_GRAPH = 1
FMT_MAX_DEGREE = 14
MAX_DEPTH = 21
_STATUS = {0: "FMT_OK", 1: "FMT_EINVAL", 2: "FMT_ENOMEM", 3: "FMT_ECUDA", 4: "FMT_ETIMEOUT", 5: "FMT_EINTERNAL"}


class FmtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class fmt_params(ctypes.Structure):
    _fields_ = [("degree", ctypes.c_int32), ("max_depth", ctypes.c_int32), ("min_pts", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("tol_rel", ctypes.c_double), ("lo", ctypes.c_double * 3),
                ("side", ctypes.c_double), ("chunk_rows", ctypes.c_int64), ("sweeps", ctypes.c_int32),
                ("options", ctypes.c_int32)]


_NL = MAX_DEPTH + 1


class fmt_stats(ctypes.Structure):
    _fields_ = [("degree", ctypes.c_int32), ("nmono", ctypes.c_int32), ("max_depth", ctypes.c_int32),
                ("n_levels", ctypes.c_int32), ("n_fitted", ctypes.c_int32), ("n_problems", ctypes.c_int32),
                ("n_points", ctypes.c_int64), ("tau", ctypes.c_double), ("maxabs_f", ctypes.c_double),
                ("nodes", ctypes.c_int64 * _NL), ("points", ctypes.c_int64 * _NL),
                ("items", ctypes.c_int64 * _NL), ("chunk_rows", ctypes.c_int64 * _NL),
                ("near_tau", ctypes.c_int64 * _NL), ("rank_flagged", ctypes.c_int64 * _NL),
                ("mixed", ctypes.c_int64 * _NL), ("mixed_points", ctypes.c_int64 * _NL)]


class fmt_request(ctypes.Structure):
    _fields_ = [("params", fmt_params), ("n", ctypes.c_int64), ("m", ctypes.c_int64),
                ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p), ("f", ctypes.c_void_p),
                ("xq", ctypes.c_void_p), ("yq", ctypes.c_void_p), ("zq", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("keep", ctypes.c_int32), ("pad", ctypes.c_int32)]


class fmt_request_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("batch_requests", ctypes.c_int32), ("batch_id", ctypes.c_int64),
                ("batch_points", ctypes.c_int64), ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double), ("resident_id", ctypes.c_int64), ("problem", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class fmt_export_header(ctypes.Structure):
    _fields_ = [("magic", ctypes.c_uint32), ("version", ctypes.c_uint32), ("degree", ctypes.c_int32),
                ("nmono", ctypes.c_int32), ("max_depth", ctypes.c_int32), ("min_pts", ctypes.c_int32),
                ("n_levels", ctypes.c_int32), ("n_fitted", ctypes.c_int32), ("has_points", ctypes.c_int32),
                ("n_problems", ctypes.c_int32), ("tol_rel", ctypes.c_double), ("tau", ctypes.c_double),
                ("maxabs_f", ctypes.c_double), ("lo", ctypes.c_double * 3), ("side", ctypes.c_double),
                ("n_points", ctypes.c_int64), ("n_nodes", ctypes.c_int64), ("level_nodes", ctypes.c_int64 * _NL)]


EXPORTED = ["fmt_nmono", "oct_build", "oct_build_batch", "fit_level", "refine", "evaluate", "evaluate_batch",
            "fmt_tree_stats", "fmt_tree_export",
            "fmt_tree_import", "fmt_tree_free", "fmt_last_error", "fmt_profile_enable", "fmt_profile_read",
            "fmt_profile_class_name", "fmt_probe_dfma", "fmt_fit_node_static", "fmt_server_create",
            "fmt_server_submit", "fmt_server_wait", "fmt_server_destroy", "fmt_server_clock", "fmt_autotune",
            "fmt_tune_get", "fmt_tune_set", "fmt_debug_fail_alloc", "fmt_wait_probe", "fmt_autotune_forest",
            "fmt_server_submit_eval", "fmt_server_release", "fmt_server_memory", "fmt_tree_trim",
            "fmt_checked_build", "fmt_check_probe", "fmt_debug_item_rows"]
STATIC_MAX_DEGREE = 8
PROFILE_CLASSES = 24


class fmt_tune_entry(ctypes.Structure):
    _fields_ = [("degree", ctypes.c_int32), ("rows", ctypes.c_int32), ("warps", ctypes.c_int32),
                ("chunk_factor", ctypes.c_int32), ("merge", ctypes.c_int32), ("source", ctypes.c_int32),
                ("sample_points", ctypes.c_int64), ("ms", ctypes.c_double), ("ms_builtin", ctypes.c_double),
                ("trials", ctypes.c_int32), ("pad", ctypes.c_int32)]


TUNE_FIELDS = ("degree", "rows", "warps", "chunk_factor", "merge", "source", "sample_points", "ms", "ms_builtin",
               "trials")


class fmt_tune_report(ctypes.Structure):
    _fields_ = [("ms_start", ctypes.c_double), ("ms_best", ctypes.c_double), ("trials", ctypes.c_int32),
                ("changed", ctypes.c_int32)]


class fmt_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * PROFILE_CLASSES), ("ms", ctypes.c_double * PROFILE_CLASSES),
                ("units", ctypes.c_double * PROFILE_CLASSES), ("flops", ctypes.c_double * PROFILE_CLASSES)]

_lock = threading.Lock()
_lib = None


def load(build: bool = True):
    """Load libfmt.so (building it with nvcc first when it is stale).

    FMT_LIBRARY names another build of the same sources to load instead
    (the sanitizer test loads an ASan/UBSan build this way, in a child
    process); it is loaded as is, never built here."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = os.environ.get("FMT_LIBRARY") or LIB_PATH
        if build and path == LIB_PATH:
            from . import build as _b
            _b.build()
        if not os.path.exists(path):
            raise ImportError("libfmt.so not found at %s; run paper_1511_01353_gb300/build.py" % path)
        L = ctypes.CDLL(path)
        P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.fmt_nmono.argtypes = [i32]
        L.fmt_nmono.restype = i32
        L.oct_build.argtypes = [ctypes.POINTER(fmt_params), i64, P, P, P, P, P, ctypes.POINTER(P)]
        L.oct_build.restype = ctypes.c_int
        L.fit_level.argtypes = [P, i32, P]
        L.fit_level.restype = ctypes.c_int
        L.refine.argtypes = [P, i32, ctypes.POINTER(i64), P]
        L.refine.restype = ctypes.c_int
        L.evaluate.argtypes = [P, i64, P, P, P, P, ctypes.POINTER(i64), P]
        L.evaluate.restype = ctypes.c_int
        L.oct_build_batch.argtypes = [ctypes.POINTER(fmt_params), i64, P, P, P, P, P, P, P, P, ctypes.POINTER(P)]
        L.oct_build_batch.restype = ctypes.c_int
        L.evaluate_batch.argtypes = [P, i64, P, P, P, P, P, ctypes.POINTER(i64), P]
        L.evaluate_batch.restype = ctypes.c_int
        L.fmt_tree_stats.argtypes = [P, ctypes.POINTER(fmt_stats)]
        L.fmt_tree_stats.restype = ctypes.c_int
        L.fmt_tree_export.argtypes = [P, P, ctypes.POINTER(ctypes.c_size_t)]
        L.fmt_tree_export.restype = ctypes.c_int
        L.fmt_tree_import.argtypes = [P, ctypes.c_size_t, P, ctypes.POINTER(P)]
        L.fmt_tree_import.restype = ctypes.c_int
        L.fmt_tree_free.argtypes = [P]
        L.fmt_tree_free.restype = None
        L.fmt_last_error.argtypes = [P]
        L.fmt_last_error.restype = ctypes.c_char_p
        L.fmt_profile_enable.argtypes = [i32]
        L.fmt_profile_enable.restype = ctypes.c_int
        L.fmt_profile_read.argtypes = [ctypes.POINTER(fmt_profile)]
        L.fmt_profile_read.restype = ctypes.c_int
        L.fmt_profile_class_name.argtypes = [i32]
        L.fmt_profile_class_name.restype = ctypes.c_char_p
        L.fmt_probe_dfma.argtypes = [i64, ctypes.POINTER(ctypes.c_double), P]
        L.fmt_probe_dfma.restype = ctypes.c_int
        L.fmt_server_create.argtypes = [i32, ctypes.c_double, i64, ctypes.POINTER(P)]
        L.fmt_server_create.restype = ctypes.c_int
        L.fmt_server_submit.argtypes = [P, ctypes.POINTER(fmt_request), ctypes.POINTER(i64)]
        L.fmt_server_submit.restype = ctypes.c_int
        L.fmt_server_wait.argtypes = [P, i64, ctypes.c_double, ctypes.POINTER(fmt_request_result)]
        L.fmt_server_wait.restype = ctypes.c_int
        L.fmt_server_destroy.argtypes = [P]
        L.fmt_server_destroy.restype = ctypes.c_int
        L.fmt_tree_trim.argtypes = [P, P]
        L.fmt_tree_trim.restype = ctypes.c_int
        L.fmt_server_submit_eval.argtypes = [P, i64, i64, P, P, P, P, ctypes.POINTER(i64)]
        L.fmt_server_submit_eval.restype = ctypes.c_int
        L.fmt_server_release.argtypes = [P, i64]
        L.fmt_server_release.restype = ctypes.c_int
        L.fmt_server_memory.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(i64)]
        L.fmt_server_memory.restype = ctypes.c_int
        L.fmt_server_clock.argtypes = []
        L.fmt_server_clock.restype = ctypes.c_double
        L.fmt_fit_node_static.argtypes = [i32, i64, P, P, P, P, P, ctypes.c_double, P, P, P, P]
        L.fmt_fit_node_static.restype = ctypes.c_int
        L.fmt_autotune.argtypes = [i32, i64, P, ctypes.POINTER(fmt_tune_entry)]
        L.fmt_autotune.restype = ctypes.c_int
        L.fmt_autotune_forest.argtypes = [P, i64, P, P, P, P, P, P, P, P, ctypes.POINTER(fmt_tune_report)]
        L.fmt_autotune_forest.restype = ctypes.c_int
        L.fmt_tune_get.argtypes = [i32, ctypes.POINTER(fmt_tune_entry)]
        L.fmt_tune_get.restype = ctypes.c_int
        L.fmt_tune_set.argtypes = [ctypes.POINTER(fmt_tune_entry)]
        L.fmt_tune_set.restype = ctypes.c_int
        L.fmt_debug_fail_alloc.argtypes = [i64]
        L.fmt_debug_fail_alloc.restype = ctypes.c_int
        L.fmt_wait_probe.argtypes = [i64, P]
        L.fmt_wait_probe.restype = ctypes.c_int
        L.fmt_checked_build.argtypes = []
        L.fmt_checked_build.restype = i32
        L.fmt_check_probe.argtypes = [i32, i32, P]
        L.fmt_check_probe.restype = ctypes.c_int
        L.fmt_debug_item_rows.argtypes = [P, i32, i64, i64, i64, P]
        L.fmt_debug_item_rows.restype = ctypes.c_int
        _lib = L
        return L


def _check(st, tree=None):
    if st != FMT_OK:
        L = load(build=False)
        msg = L.fmt_last_error(tree.handle if tree is not None else None)
        raise FmtError(st, msg.decode() if msg else "")


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptrs(stream, *specs):
    """Device pointers of caller-owned tensors, checked before the library
    sees them (the library cannot check a device buffer's size).

    Each spec is (tensor, name, dtype, count, exact): a contiguous torch
    tensor of that dtype with exactly `count` elements (at least `count` when
    `exact` is False, for outputs), on the CUDA device the call runs on (the
    stream's, else the current device).  A wrong type, dtype, layout or
    device raises TypeError; a wrong size FmtError(FMT_EINVAL).  Sizes are
    checked first, then the device."""
    import torch
    for t, name, dtype, count, exact in specs:
        if not isinstance(t, torch.Tensor):
            raise TypeError("%s must be a torch tensor" % name)
        if t.dtype != dtype or not t.is_contiguous():
            raise TypeError("%s must be a contiguous %s tensor" % (name, str(dtype).replace("torch.", "")))
        k = t.numel()
        if (k != count) if exact else (k < count):
            raise FmtError(FMT_EINVAL, "%s has %d elements; %s %d" % (name, k, "expected" if exact else
                                                                       "needs at least", count))
    for t, name, *_ in specs:
        if not t.is_cuda:
            raise TypeError("%s must be a CUDA tensor" % name)
    sdev = getattr(stream, "device", None) if stream is not None else None
    dev = sdev.index if sdev is not None else torch.cuda.current_device()
    for t, name, *_ in specs:
        if t.device.index != dev:
            raise TypeError("%s is on %s, the call runs on cuda:%d" % (name, t.device, dev))
    return [ctypes.c_void_p(t.data_ptr()) for t, *_ in specs]


def _f64(n, **named):
    """_ptrs specs of float64 buffers of exactly n elements, in keyword order."""
    import torch
    return [(t, name, torch.float64, n, True) for name, t in named.items()]


def _numel(t, name):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % name)
    return int(t.numel())


class Tree:
    """Owning handle of an fmt_tree (freed on close() or garbage collection)."""

    def __init__(self, handle):
        self.handle = handle

    def close(self):
        if self.handle:
            load(build=False).fmt_tree_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_params(degree, max_depth, min_pts, tol_rel, lo=(0.0, 0.0, 0.0), side=1.0, chunk_rows=0,
                precision=FMT_FP64, sweeps=0, graph=False):
    """fmt_params; precision FMT_FP64 or FMT_MIXED, sweeps (mixed only): 0 = 3, -1 = none;
    graph: capture each fit_level in a CUDA graph (FMT_OPT_GRAPH)."""
    p = fmt_params()
    p.degree, p.max_depth, p.min_pts, p.precision = degree, max_depth, min_pts, precision
    p.sweeps = sweeps
    p.options = FMT_OPT_GRAPH if graph else 0
    p.tol_rel = tol_rel
    for a in range(3):
        p.lo[a] = lo[a]
    p.side = side
    p.chunk_rows = chunk_rows
    return p


def fmt_nmono(degree: int) -> int:
    return int(load().fmt_nmono(degree))


def oct_build(params: fmt_params, x, y, z, f, stream=None) -> Tree:
    n = _numel(x, "x")
    px, py, pz, pf = _ptrs(stream, *_f64(n, x=x, y=y, z=z, f=f))
    L = load()
    h = ctypes.c_void_p()
    st = L.oct_build(ctypes.byref(params), n, px, py, pz, pf, _stream_handle(stream), ctypes.byref(h))
    _check(st)
    return Tree(h)


def oct_build_batch(params: fmt_params, offsets, x, y, z, f, degrees=None, boxes=None, stream=None) -> Tree:
    """Forest of independent problems: offsets (n_problems+1, host), per-problem
    degrees (host int32) and boxes (host, 4 per problem: lo x, lo y, lo z, side)."""
    off = np.ascontiguousarray(offsets, dtype=np.int64).reshape(-1)
    if off.shape[0] < 2:
        raise FmtError(FMT_EINVAL, "offsets needs n_problems + 1 >= 2 entries")
    n_prob = int(off.shape[0] - 1)
    deg = None if degrees is None else np.ascontiguousarray(degrees, dtype=np.int32).reshape(-1)
    box = None if boxes is None else np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1)
    if deg is not None and deg.shape[0] != n_prob:
        raise FmtError(FMT_EINVAL, "degrees has %d entries; expected %d" % (deg.shape[0], n_prob))
    if box is not None and box.shape[0] != 4 * n_prob:
        raise FmtError(FMT_EINVAL, "boxes has %d values; expected 4 per problem (%d)" % (box.shape[0], 4 * n_prob))
    px, py, pz, pf = _ptrs(stream, *_f64(int(off[-1]), x=x, y=y, z=z, f=f))
    L = load()
    h = ctypes.c_void_p()
    st = L.oct_build_batch(ctypes.byref(params), n_prob, off.ctypes.data_as(ctypes.c_void_p),
                           None if deg is None else deg.ctypes.data_as(ctypes.c_void_p),
                           None if box is None else box.ctypes.data_as(ctypes.c_void_p),
                           px, py, pz, pf, _stream_handle(stream), ctypes.byref(h))
    _check(st)
    return Tree(h)


def fit_level(tree: Tree, depth: int, stream=None):
    _check(load().fit_level(tree.handle, depth, _stream_handle(stream)), tree)


def refine(tree: Tree, depth: int, stream=None) -> int:
    n = ctypes.c_int64(0)
    _check(load().refine(tree.handle, depth, ctypes.byref(n), _stream_handle(stream)), tree)
    return int(n.value)


def evaluate(tree: Tree, xq, yq, zq, out, count_outside=False, stream=None):
    import torch
    m = _numel(xq, "xq")
    px, py, pz, po = _ptrs(stream, *_f64(m, xq=xq, yq=yq, zq=zq), (out, "out", torch.float64, m, False))
    nout = ctypes.c_int64(0)
    st = load().evaluate(tree.handle, m, px, py, pz, po, ctypes.byref(nout) if count_outside else None,
                         _stream_handle(stream))
    _check(st, tree)
    return int(nout.value) if count_outside else None


def evaluate_batch(tree: Tree, target_problem, xq, yq, zq, out, count_outside=False, stream=None):
    """target_problem: int32 CUDA tensor with the problem index of every target."""
    import torch
    m = _numel(xq, "xq")
    px, py, pz, pt, po = _ptrs(stream, *_f64(m, xq=xq, yq=yq, zq=zq),
                               (target_problem, "target_problem", torch.int32, m, True),
                               (out, "out", torch.float64, m, False))
    nout = ctypes.c_int64(0)
    st = load().evaluate_batch(tree.handle, m, pt, px, py, pz, po, ctypes.byref(nout) if count_outside else None,
                               _stream_handle(stream))
    _check(st, tree)
    return int(nout.value) if count_outside else None


def fmt_tree_stats(tree: Tree) -> fmt_stats:
    s = fmt_stats()
    _check(load().fmt_tree_stats(tree.handle, ctypes.byref(s)), tree)
    return s


def fmt_tree_export(tree: Tree) -> bytes:
    L = load()
    n = ctypes.c_size_t(0)
    _check(L.fmt_tree_export(tree.handle, None, ctypes.byref(n)), tree)
    buf = (ctypes.c_char * n.value)()
    _check(L.fmt_tree_export(tree.handle, ctypes.cast(buf, ctypes.c_void_p), ctypes.byref(n)), tree)
    return bytes(buf)


def fmt_tree_import(blob: bytes, stream=None) -> Tree:
    L = load()
    h = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(L.fmt_tree_import(ctypes.cast(buf, ctypes.c_void_p), len(blob), _stream_handle(stream), ctypes.byref(h)))
    return Tree(h)


def fmt_profile_enable(on: bool):
    _check(load().fmt_profile_enable(1 if on else 0))


def fmt_profile_read() -> dict:
    """{class name: dict(launches, ms, units, flops)} for the classes the library defines."""
    L = load()
    p = fmt_profile()
    _check(L.fmt_profile_read(ctypes.byref(p)))
    out = {}
    for k in range(PROFILE_CLASSES):
        name = L.fmt_profile_class_name(k)
        if not name:
            break
        out[name.decode()] = dict(launches=int(p.launches[k]), ms=float(p.ms[k]), units=float(p.units[k]),
                                  flops=float(p.flops[k]))
    return out


def fmt_probe_dfma(iters: int = 20000, stream=None) -> float:
    """Measured FP64 FMA rate of the current GPU (DFMA per second)."""
    v = ctypes.c_double(0.0)
    _check(load().fmt_probe_dfma(iters, ctypes.byref(v), _stream_handle(stream)))
    return float(v.value)


def _entry_dict(e: fmt_tune_entry) -> dict:
    return {k: getattr(e, k) for k in TUNE_FIELDS}


def fmt_autotune(degree: int, sample_points: int = 0, stream=None) -> dict:
    """Time QR launch configurations for `degree` and install the fastest (synchronises)."""
    e = fmt_tune_entry()
    _check(load().fmt_autotune(degree, sample_points, _stream_handle(stream), ctypes.byref(e)))
    return _entry_dict(e)


def fmt_autotune_forest(params: fmt_params, offsets, x, y, z, f, degrees=None, boxes=None, stream=None) -> dict:
    """Tune the per-degree QR table on a forest (a sample of the one about to be
    fitted) by timing its whole level loop (synchronises); returns the report."""
    off = np.ascontiguousarray(offsets, dtype=np.int64).reshape(-1)
    if off.shape[0] < 2:
        raise FmtError(FMT_EINVAL, "offsets needs n_problems + 1 >= 2 entries")
    n_prob = int(off.shape[0] - 1)
    deg = None if degrees is None else np.ascontiguousarray(degrees, dtype=np.int32).reshape(-1)
    box = None if boxes is None else np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1)
    if deg is not None and deg.shape[0] != n_prob:
        raise FmtError(FMT_EINVAL, "degrees has %d entries; expected %d" % (deg.shape[0], n_prob))
    if box is not None and box.shape[0] != 4 * n_prob:
        raise FmtError(FMT_EINVAL, "boxes has %d values; expected 4 per problem (%d)" % (box.shape[0], 4 * n_prob))
    px, py, pz, pf = _ptrs(stream, *_f64(int(off[-1]), x=x, y=y, z=z, f=f))
    rep = fmt_tune_report()
    _check(load().fmt_autotune_forest(ctypes.byref(params), n_prob, off.ctypes.data_as(ctypes.c_void_p),
                                      None if deg is None else deg.ctypes.data_as(ctypes.c_void_p),
                                      None if box is None else box.ctypes.data_as(ctypes.c_void_p),
                                      px, py, pz, pf, _stream_handle(stream), ctypes.byref(rep)))
    return {"ms_start": rep.ms_start, "ms_best": rep.ms_best, "trials": int(rep.trials), "changed": int(rep.changed)}


def fmt_tune_get(degree: int) -> dict:
    """The QR launch configuration in force for `degree` (host only)."""
    e = fmt_tune_entry()
    _check(load().fmt_tune_get(degree, ctypes.byref(e)))
    return _entry_dict(e)


def fmt_tune_set(entry: dict):
    """Install a configuration (e.g. saved from fmt_autotune); source 0 restores the built-in rule."""
    e = fmt_tune_entry()
    for k in TUNE_FIELDS:
        if k in entry:
            setattr(e, k, entry[k])
    if "source" not in entry:
        e.source = 2
    _check(load().fmt_tune_set(ctypes.byref(e)))


def fmt_debug_fail_alloc(k: int):
    """Make the k-th device allocation of the library from now fail (FMT_ENOMEM); 0 disarms."""
    _check(load().fmt_debug_fail_alloc(k))


def fmt_wait_probe(limit_ns: int, stream=None):
    """Bounded wait that nothing satisfies; raises FmtError(FMT_ETIMEOUT) when the bound runs out."""
    _check(load().fmt_wait_probe(limit_ns, _stream_handle(stream)))


def fmt_checked_build() -> bool:
    """True when the loaded library was built with device bounds checks (-DFMT_CHECKED)."""
    return bool(load().fmt_checked_build())


def fmt_check_probe(i: int, n: int, stream=None):
    """Self-test of the device bounds checks: element i of a 64-element device
    array, written when i < n passes the checked build's test.  Raises
    FmtError(FMT_EINTERNAL) for i >= n in the checked build."""
    _check(load().fmt_check_probe(i, n, _stream_handle(stream)))


def fmt_debug_item_rows(tree: "Tree", depth: int, item: int, start: int, end: int, stream=None):
    """Test hook: set one work item's row range (0 <= start <= end <= n) of
    the planned level awaiting its fit."""
    _check(load().fmt_debug_item_rows(tree.handle, depth, item, start, end, _stream_handle(stream)), tree)


def fmt_fit_node_static(degree: int, x, y, z, r_in, coef, r_out, flags=None, lo=(0.0, 0.0, 0.0), side=1.0,
                        stream=None):
    """Allocation-free fit of one point set in the root frame of [lo, lo+side)^3.

    All buffers are caller-owned CUDA tensors: coef (nmono(degree) float64)
    and r_out (n float64) are written; flags, if given, is a 1-element int32
    CUDA tensor.  The library allocates nothing for this call."""
    import torch
    lo_a = (ctypes.c_double * 3)(*lo)
    n = _numel(x, "x")
    ncoef = fmt_nmono(degree) if degree >= 0 else 0
    if _numel(coef, "coef") < ncoef:
        raise FmtError(FMT_EINVAL, "coef has %d elements; degree %d needs %d" % (coef.numel(), degree, ncoef))
    specs = _f64(n, x=x, y=y, z=z, r_in=r_in) + [(coef, "coef", torch.float64, ncoef, False),
                                                  (r_out, "r_out", torch.float64, n, False)]
    if flags is not None:
        specs.append((flags, "flags", torch.int32, 1, False))
    ptrs = _ptrs(stream, *specs)
    px, py, pz, pr, pc, po = ptrs[:6]
    fp = ptrs[6] if flags is not None else None
    st = load().fmt_fit_node_static(degree, n, px, py, pz, pr, ctypes.cast(lo_a, ctypes.c_void_p), side, pc, po,
                                    fp, _stream_handle(stream))
    _check(st)


def fmt_profile_class_name(k: int):
    n = load().fmt_profile_class_name(k)
    return n.decode() if n else None


def fmt_tree_trim(tree: Tree, stream=None):
    """Free the fit-only scratch of a tree kept for evaluation."""
    _check(load().fmt_tree_trim(tree.handle, _stream_handle(stream)), tree)


def fmt_tree_free(tree: Tree):
    tree.close()


def fmt_last_error(tree: Tree | None = None) -> str:
    msg = load().fmt_last_error(tree.handle if tree is not None else None)
    return msg.decode() if msg else ""


# ----------------------------------------------------------------- helpers
def fit_all(tree: Tree, stream=None) -> Tree:
    """The driver loop after oct_build: for depth 0, 1, ...: fit_level, then
    refine until it creates no node."""
    d = 0
    while True:
        fit_level(tree, d, stream)
        if refine(tree, d, stream) == 0:
            break
        d += 1
    return tree


def fit(params: fmt_params, x, y, z, f, stream=None) -> Tree:
    """oct_build followed by the driver loop of fit_level / refine."""
    return fit_all(oct_build(params, x, y, z, f, stream), stream)


@dataclasses.dataclass
class ExportedTree:
    header: dict
    prefix: np.ndarray      # node keys: problem << 3*depth | Morton prefix
    start: np.ndarray
    count: np.ndarray
    depth: np.ndarray
    flags: np.ndarray
    deg_used: np.ndarray
    refine_mask: np.ndarray
    near_mask: np.ndarray
    problem: np.ndarray
    child_E: np.ndarray
    child_n: np.ndarray
    coef: np.ndarray
    problems: dict          # degree, q_root, tau, maxabs, lo [P,3], side, start, count
    code: np.ndarray | None
    perm: np.ndarray | None
    resid: np.ndarray | None

    def morton_prefix(self):
        """Node keys with the problem bits removed."""
        d = self.depth.astype(np.uint64)
        mask = np.where(d > 0, (np.uint64(1) << (np.uint64(3) * d)) - np.uint64(1), np.uint64(0))
        return self.prefix & mask


def parse_export(blob: bytes) -> ExportedTree:
    H = fmt_export_header.from_buffer_copy(blob[:ctypes.sizeof(fmt_export_header)])
    if H.magic != 0x32544D46 or H.version != 2:
        raise ValueError("not an FMT2 blob")
    hdr = {name: getattr(H, name) for name, _ in fmt_export_header._fields_}
    hdr["lo"] = tuple(H.lo)
    hdr["level_nodes"] = list(H.level_nodes)
    K, nm, N, P = H.n_nodes, H.nmono, H.n_points if H.has_points else 0, H.n_problems
    off = ctypes.sizeof(fmt_export_header)

    def take(dtype, count):
        nonlocal off
        a = np.frombuffer(blob, dtype=dtype, count=count, offset=off).copy()
        off += a.nbytes
        return a

    prefix = take(np.uint64, K)
    start = take(np.int64, K)
    count = take(np.int64, K)
    depth = take(np.int32, K)
    flags = take(np.int32, K)
    deg = take(np.int32, K)
    masks = take(np.int32, K)
    prob = take(np.int32, K)
    take(np.int32, K)
    cE = take(np.float64, 8 * K).reshape(K, 8)
    cn = take(np.int64, 8 * K).reshape(K, 8)
    coef = take(np.float64, nm * K).reshape(K, nm)
    problems = dict(degree=take(np.int32, P), q_root=take(np.int32, P), tau=take(np.float64, P),
                    maxabs=take(np.float64, P), lo=take(np.float64, 3 * P).reshape(P, 3), side=take(np.float64, P),
                    start=take(np.int64, P), count=take(np.int64, P))
    code = perm = resid = None
    if H.has_points:
        code = take(np.uint64, N)
        perm = take(np.int64, N)
        resid = take(np.float64, N)
    return ExportedTree(hdr, prefix, start, count, depth, flags, deg, masks & 0xFF, (masks >> 8) & 0xFF, prob, cE,
                        cn, coef, problems, code, perm, resid)


def build_export(header: dict, prefix, depth, flags, deg_used, child_E, child_n, coef, start=None, count=None,
                 refine_mask=None, near_mask=None) -> bytes:
    """Serialise the node arrays of a single-problem tree into an FMT2 blob (no
    per-point arrays), e.g. to upload a tree built elsewhere for evaluation
    through fmt_tree_import.  prefix holds Morton prefixes (problem 0)."""
    K = int(prefix.shape[0])
    H = fmt_export_header()
    H.magic, H.version = 0x32544D46, 2
    H.degree, H.nmono = header["degree"], header["nmono"]
    H.max_depth, H.min_pts = header["max_depth"], header["min_pts"]
    lv = np.bincount(np.asarray(depth, dtype=np.int64), minlength=1)
    H.n_levels = H.n_fitted = int(lv.shape[0])
    H.has_points = 0
    H.n_problems = 1
    H.tol_rel, H.tau, H.maxabs_f = header["tol_rel"], header["tau"], header["maxabs_f"]
    for a in range(3):
        H.lo[a] = header["lo"][a]
    H.side = header["side"]
    H.n_points = header.get("n_points", 0)
    H.n_nodes = K
    for d in range(lv.shape[0]):
        H.level_nodes[d] = int(lv[d])
    z64 = np.zeros(K, np.int64)
    z32 = np.zeros(K, np.int32)
    rm = z32 if refine_mask is None else np.asarray(refine_mask, np.int32)
    nm_ = z32 if near_mask is None else np.asarray(near_mask, np.int32)
    n_pts = int(header.get("n_points", 0))
    parts = [bytes(H), np.asarray(prefix, np.uint64).tobytes(),
             (z64 if start is None else np.asarray(start, np.int64)).tobytes(),
             (z64 if count is None else np.asarray(count, np.int64)).tobytes(),
             np.asarray(depth, np.int32).tobytes(), np.asarray(flags, np.int32).tobytes(),
             np.asarray(deg_used, np.int32).tobytes(), (rm | (nm_ << 8)).astype(np.int32).tobytes(),
             z32.tobytes(), z32.tobytes(),
             np.asarray(child_E, np.float64).tobytes(), np.asarray(child_n, np.int64).tobytes(),
             np.asarray(coef, np.float64).tobytes(),
             np.array([header["degree"]], np.int32).tobytes(), np.array([header["degree"]], np.int32).tobytes(),
             np.array([header["tau"]], np.float64).tobytes(), np.array([header["maxabs_f"]], np.float64).tobytes(),
             np.asarray(header["lo"], np.float64).tobytes(), np.array([header["side"]], np.float64).tobytes(),
             np.array([0], np.int64).tobytes(), np.array([n_pts], np.int64).tobytes()]
    return b"".join(parts)


class Server:
    """The serving engine (fmt_server_*): submit fit+evaluate requests with
    host arrays, wait for their results.  Arrays are kept referenced here
    until the request is returned by wait()."""

    def __init__(self, slots=2, budget_bytes=150e9, max_batch_points=4_000_000):
        L = load()
        h = ctypes.c_void_p()
        _check(L.fmt_server_create(slots, float(budget_bytes), int(max_batch_points), ctypes.byref(h)))
        self.handle = h
        self._live = {}

    @staticmethod
    def clock():
        return float(load().fmt_server_clock())

    def submit(self, params: fmt_params, x, y, z, f, xq=None, yq=None, zq=None, keep=False) -> int:
        arr = [np.ascontiguousarray(a, dtype=np.float64).reshape(-1) for a in (x, y, z, f)]
        if xq is None and (yq is not None or zq is not None):
            raise FmtError(FMT_EINVAL, "targets need all of xq, yq, zq")
        q = [np.ascontiguousarray(a, dtype=np.float64).reshape(-1) for a in (xq, yq, zq)] if xq is not None else \
            [np.zeros(0) for _ in range(3)]
        for name, a in zip(("y", "z", "f"), arr[1:]):
            if a.shape[0] != arr[0].shape[0]:
                raise FmtError(FMT_EINVAL, "%s has %d points; x has %d" % (name, a.shape[0], arr[0].shape[0]))
        for name, a in zip(("yq", "zq"), q[1:]):
            if a.shape[0] != q[0].shape[0]:
                raise FmtError(FMT_EINVAL, "%s has %d targets; xq has %d" % (name, a.shape[0], q[0].shape[0]))
        out = np.empty(q[0].shape[0], dtype=np.float64)
        r = fmt_request()
        r.params = params
        r.n, r.m = arr[0].shape[0], q[0].shape[0]
        r.x, r.y, r.z, r.f = (a.ctypes.data for a in arr)
        r.xq, r.yq, r.zq = (a.ctypes.data if a.shape[0] else None for a in q)
        r.out = out.ctypes.data if out.shape[0] else None
        r.keep = 1 if keep else 0
        t = ctypes.c_int64()
        _check(load().fmt_server_submit(self.handle, ctypes.byref(r), ctypes.byref(t)))
        self._live[t.value] = (arr, q, out)
        return t.value

    def submit_eval(self, resident_id: int, xq, yq, zq) -> int:
        """Evaluate-only request against a tree kept by submit(..., keep=True)."""
        q = [np.ascontiguousarray(a, dtype=np.float64).reshape(-1) for a in (xq, yq, zq)]
        for name, a in zip(("yq", "zq"), q[1:]):
            if a.shape[0] != q[0].shape[0]:
                raise FmtError(FMT_EINVAL, "%s has %d targets; xq has %d" % (name, a.shape[0], q[0].shape[0]))
        out = np.empty(q[0].shape[0], dtype=np.float64)
        m = q[0].shape[0]
        t = ctypes.c_int64()
        _check(load().fmt_server_submit_eval(self.handle, int(resident_id), m,
                                             *(a.ctypes.data if m else None for a in q),
                                             out.ctypes.data if m else None, ctypes.byref(t)))
        self._live[t.value] = (None, q, out)
        return t.value

    def release(self, resident_id: int):
        _check(load().fmt_server_release(self.handle, int(resident_id)))

    def memory(self) -> dict:
        """Bytes admitted now (running batches and resident trees), their peak, resident trees."""
        a, p, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        _check(load().fmt_server_memory(self.handle, ctypes.byref(a), ctypes.byref(p), ctypes.byref(n)))
        return {"admitted": a.value, "peak_admitted": p.value, "resident_trees": int(n.value)}

    def wait(self, ticket: int, timeout: float = -1.0):
        """(values at the targets, result dict) of a submitted request."""
        res = fmt_request_result()
        _check(load().fmt_server_wait(self.handle, ticket, float(timeout), ctypes.byref(res)))
        arr, q, out = self._live.pop(ticket)
        info = {name: getattr(res, name) for name, _ in fmt_request_result._fields_}
        return out, info

    def close(self):
        if self.handle is not None and self.handle.value:
            load().fmt_server_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
