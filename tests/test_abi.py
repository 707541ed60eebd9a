"""Host-side checks of the C ABI: libfmt.so builds for sm_103a, exports every
function include/fmt.h declares, the ctypes structures match the C layout,
and argument validation answers before any device work."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

from paper_1511_01353_gb300 import fmt as F

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fmt.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([A-Za-z_][A-Za-z0-9_]*)\s*\(", src, re.M)
    return sorted(set(names))


def test_header_declares_the_four_calls():
    names = declared_functions()
    for n in ("oct_build", "fit_level", "refine", "evaluate"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = F.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(F.EXPORTED) == declared_functions()


def test_checked_build_compiles_and_exports_the_same_symbols():
    # the bounds-checked build (-DFMT_CHECKED) of the same sources; host-only
    # calls, no GPU needed
    from paper_1511_01353_gb300 import build as B
    lib = ctypes.CDLL(B.build_checked())
    for name in declared_functions():
        assert hasattr(lib, name), name
    lib.fmt_checked_build.restype = ctypes.c_int32
    assert lib.fmt_checked_build() == 1
    assert not F.fmt_checked_build()


def _c_layout():
    code = r'''
#include <stdio.h>
#include <stddef.h>
#include "fmt.h"
int main(void){
  printf("%zu %zu %zu %zu %zu\n", sizeof(fmt_params), offsetof(fmt_params, tol_rel), offsetof(fmt_params, side),
         offsetof(fmt_params, chunk_rows), sizeof(fmt_stats));
  printf("%zu %zu %zu\n", sizeof(fmt_export_header), offsetof(fmt_export_header, tol_rel),
         offsetof(fmt_export_header, level_nodes));
  printf("%zu %zu %zu %zu\n", offsetof(fmt_params, sweeps), offsetof(fmt_stats, mixed),
         offsetof(fmt_stats, mixed_points), sizeof(fmt_profile));
  printf("%zu %zu %zu %zu %zu\n", offsetof(fmt_params, options), sizeof(fmt_tune_entry),
         offsetof(fmt_tune_entry, sample_points), offsetof(fmt_tune_entry, ms_builtin),
         offsetof(fmt_tune_entry, trials));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(c, "w").write(code)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    return [int(v) for v in out]


def test_struct_layouts_match_c():
    v = _c_layout()
    assert v[0] == ctypes.sizeof(F.fmt_params)
    assert v[1] == F.fmt_params.tol_rel.offset
    assert v[2] == F.fmt_params.side.offset
    assert v[3] == F.fmt_params.chunk_rows.offset
    assert v[4] == ctypes.sizeof(F.fmt_stats)
    assert v[5] == ctypes.sizeof(F.fmt_export_header)
    assert v[6] == F.fmt_export_header.tol_rel.offset
    assert v[7] == F.fmt_export_header.level_nodes.offset
    assert v[8] == F.fmt_params.sweeps.offset
    assert v[9] == F.fmt_stats.mixed.offset
    assert v[10] == F.fmt_stats.mixed_points.offset
    assert v[11] == ctypes.sizeof(F.fmt_profile)
    assert v[12] == F.fmt_params.options.offset
    assert v[13] == ctypes.sizeof(F.fmt_tune_entry)
    assert v[14] == F.fmt_tune_entry.sample_points.offset
    assert v[15] == F.fmt_tune_entry.ms_builtin.offset
    assert v[16] == F.fmt_tune_entry.trials.offset


def test_tune_table_is_host_only_and_checks_entries():
    # built-in rule: 64-row blocks while two CTAs fit (ld(166) = 180), 32 rows
    # for degree 14 (ld(681) = 692), 4 warps below degree 8 and 8 from it on,
    # chunks of 4 m rows, packed merge
    e = F.fmt_tune_get(8)
    assert (e["source"], e["rows"], e["warps"], e["chunk_factor"], e["merge"]) == (0, 64, 8, 4, 0)
    assert F.fmt_tune_get(7)["warps"] == 4
    assert F.fmt_tune_get(14)["rows"] == 32
    F.fmt_tune_set(dict(degree=8, rows=16, warps=8, chunk_factor=2, merge=1))
    try:
        g = F.fmt_tune_get(8)
        assert (g["source"], g["rows"], g["warps"], g["chunk_factor"], g["merge"]) == (2, 16, 8, 2, 1)
        assert F.fmt_tune_get(7)["source"] == 0  # other degrees untouched
        good = dict(degree=8, rows=32, warps=4, chunk_factor=4, merge=0)
        for k, v in (("rows", 40), ("warps", 6), ("chunk_factor", 3), ("merge", 2), ("degree", 15),
                     ("degree", -1)):
            with pytest.raises(F.FmtError):
                F.fmt_tune_set(dict(good, **{k: v}))
        with pytest.raises(F.FmtError):  # 66 rows x 692 doubles exceed 227 KB
            F.fmt_tune_set(dict(degree=14, rows=64, warps=4, chunk_factor=4, merge=0))
        assert F.fmt_tune_get(8)["rows"] == 16  # a rejected entry changes nothing
    finally:
        F.fmt_tune_set(dict(degree=8, source=0))
    assert F.fmt_tune_get(8)["source"] == 0


def test_nmono_matches_paper_values():
    assert [F.fmt_nmono(p) for p in (6, 10, 14)] == [84, 286, 680]
    assert F.fmt_nmono(-1) == 0


@pytest.mark.parametrize("field,value", [("degree", 15), ("degree", -1), ("max_depth", 22), ("min_pts", -3),
                                         ("tol_rel", -1.0), ("tol_rel", float("nan")), ("side", 0.0),
                                         ("precision", 2), ("precision", -1), ("chunk_rows", -64),
                                         ("sweeps", 4), ("sweeps", -2), ("options", 2),
                                         ("options", -1)])
def test_oct_build_rejects_bad_params_before_device_work(field, value):
    lib = F.load()
    p = F.make_params(4, 3, 64, 1e-4)
    setattr(p, field, value)
    h = ctypes.c_void_p()
    st = lib.oct_build(ctypes.byref(p), 10, ctypes.c_void_p(8), ctypes.c_void_p(8), ctypes.c_void_p(8),
                       ctypes.c_void_p(8), None, ctypes.byref(h))
    assert st == F.FMT_EINVAL
    assert not h.value
    assert F.fmt_last_error()


def test_oct_build_rejects_empty_and_null():
    lib = F.load()
    p = F.make_params(4, 3, 64, 1e-4)
    h = ctypes.c_void_p()
    assert lib.oct_build(ctypes.byref(p), 0, None, None, None, None, None, ctypes.byref(h)) == F.FMT_EINVAL
    assert lib.oct_build(ctypes.byref(p), 5, None, None, None, None, None, ctypes.byref(h)) == F.FMT_EINVAL
    assert lib.oct_build(None, 5, None, None, None, None, None, ctypes.byref(h)) == F.FMT_EINVAL


def test_calls_on_null_tree_fail_cleanly():
    lib = F.load()
    n = ctypes.c_int64(7)
    assert lib.fit_level(None, 0, None) == F.FMT_EINVAL
    assert lib.refine(None, 0, ctypes.byref(n), None) == F.FMT_EINVAL
    assert lib.evaluate(None, 0, None, None, None, None, None, None) == F.FMT_EINVAL
    assert lib.fmt_debug_item_rows(None, 0, 0, 0, 1, None) == F.FMT_EINVAL
    lib.fmt_tree_free(None)


def test_check_probe_rejects_indices_outside_its_array():
    lib = F.load()
    for i, n in ((64, 8), (-1, 8), (3, 33), (3, -1)):
        assert lib.fmt_check_probe(i, n, None) == F.FMT_EINVAL


def test_import_rejects_garbage():
    lib = F.load()
    h = ctypes.c_void_p()
    junk = ctypes.create_string_buffer(b"\0" * 512, 512)
    assert lib.fmt_tree_import(junk, 512, None, ctypes.byref(h)) == F.FMT_EINVAL
    assert lib.fmt_tree_import(junk, 8, None, ctypes.byref(h)) == F.FMT_EINVAL


def test_failure_diagnostics_check_arguments_on_the_host():
    lib = F.load()
    assert lib.fmt_debug_fail_alloc(-1) == F.FMT_EINVAL
    assert lib.fmt_debug_fail_alloc(0) == F.FMT_OK
    assert lib.fmt_wait_probe(10, None) == F.FMT_EINVAL  # bound below 1 us
    assert lib.fmt_wait_probe(10 ** 11, None) == F.FMT_EINVAL


def test_binding_checks_buffer_sizes_before_any_call():
    # The library cannot see the size of a device buffer, so the binding
    # checks every tensor against the counts the call passes: a short buffer
    # would otherwise be read or written out of bounds on the device.
    torch = pytest.importorskip("torch")
    v = lambda n, dt=torch.float64: torch.zeros(n, dtype=dt)  # noqa: E731
    p = F.make_params(2, 3, 10, 1e-4)
    with pytest.raises(F.FmtError) as e:
        F.oct_build(p, v(6), v(5), v(6), v(6))
    assert e.value.status == F.FMT_EINVAL and "y has 5 elements" in str(e.value)
    with pytest.raises(F.FmtError):
        F.oct_build(p, v(6), v(6), v(6), v(7))
    with pytest.raises(TypeError, match="CUDA"):  # right sizes: then the device is checked
        F.oct_build(p, v(6), v(6), v(6), v(6))
    with pytest.raises(TypeError, match="float64"):
        F.oct_build(p, v(6), v(6, torch.float32), v(6), v(6))
    with pytest.raises(TypeError, match="contiguous"):
        F.oct_build(p, v(6), v(12)[::2], v(6), v(6))
    with pytest.raises(TypeError):
        F.oct_build(p, [0.0] * 6, v(6), v(6), v(6))

    x = v(100)
    with pytest.raises(F.FmtError, match="expected 90"):  # offsets end short of the buffers
        F.oct_build_batch(p, [0, 40, 90], x, x, x, x)
    with pytest.raises(F.FmtError, match="degrees"):
        F.oct_build_batch(p, [0, 40, 100], x, x, x, x, degrees=[3])
    with pytest.raises(F.FmtError, match="boxes"):
        F.oct_build_batch(p, [0, 40, 100], x, x, x, x, boxes=[0.0, 0.0, 0.0, 1.0])
    with pytest.raises(F.FmtError, match="offsets"):
        F.oct_build_batch(p, [0], x, x, x, x)

    t = F.Tree(None)  # never reached: the checks come first
    with pytest.raises(F.FmtError, match="out has 9 elements"):
        F.evaluate(t, v(10), v(10), v(10), v(9))
    with pytest.raises(F.FmtError, match="zq"):
        F.evaluate(t, v(10), v(10), v(11), v(10))
    with pytest.raises(TypeError, match="CUDA"):  # a larger output buffer is allowed
        F.evaluate(t, v(10), v(10), v(10), v(12))
    with pytest.raises(F.FmtError, match="target_problem"):
        F.evaluate_batch(t, v(9, torch.int32), v(10), v(10), v(10), v(10))
    with pytest.raises(TypeError, match="int32"):
        F.evaluate_batch(t, v(10, torch.int64), v(10), v(10), v(10), v(10))

    with pytest.raises(F.FmtError, match="degree 4 needs 35"):
        F.fmt_fit_node_static(4, v(50), v(50), v(50), v(50), v(34), v(50))
    with pytest.raises(F.FmtError, match="r_out"):
        F.fmt_fit_node_static(4, v(50), v(50), v(50), v(50), v(35), v(49))
    with pytest.raises(F.FmtError, match="r_in"):
        F.fmt_fit_node_static(4, v(50), v(50), v(50), v(51), v(35), v(50))
    with pytest.raises(F.FmtError, match="flags"):
        F.fmt_fit_node_static(4, v(50), v(50), v(50), v(50), v(35), v(50), flags=v(0, torch.int32))


def test_server_submit_checks_host_array_sizes():
    srv = object.__new__(F.Server)  # no engine: the checks come before the call
    srv.handle, srv._live = None, {}
    p = F.make_params(2, 3, 10, 1e-4)
    a = np.zeros(8)
    with pytest.raises(F.FmtError, match="f has 7 points"):
        srv.submit(p, a, a, a, np.zeros(7))
    with pytest.raises(F.FmtError, match="zq has 3 targets"):
        srv.submit(p, a, a, a, a, np.zeros(4), np.zeros(4), np.zeros(3))
    with pytest.raises(F.FmtError, match="all of xq"):
        srv.submit(p, a, a, a, a, None, np.zeros(4), np.zeros(4))


def _oracle_blob():
    # an FMT2 blob of a small three-level oracle tree, as a caller would
    # serialise a tree built elsewhere (no device involved)
    from oracle import oracle as O
    from tests import treecmp as TC
    rng = np.random.default_rng(41)
    x, y, z = rng.uniform(0, 1, (3, 1500))
    T = O.fit(x, y, z, np.sin(3 * x) + y * z, 2, 2, 10, 1e-4)
    pref = (TC.spread3(T.ixyz[:, 0]) | (TC.spread3(T.ixyz[:, 1]) << np.uint64(1)) |
            (TC.spread3(T.ixyz[:, 2]) << np.uint64(2)))
    order = np.lexsort((pref, T.depth))
    hdr = dict(degree=T.degree, nmono=T.nmono, max_depth=T.max_depth, min_pts=T.min_pts, tol_rel=T.tol_rel,
               tau=T.tau, maxabs_f=T.maxabs, lo=T.lo, side=T.side, n_points=x.shape[0])
    blob = F.build_export(hdr, pref[order], T.depth[order], T.flags[order], T.deg_used[order], T.child_E[order],
                          T.child_n[order], T.coef[order])
    return T, blob


def test_import_validates_the_blob_before_touching_the_device():
    # fmt_tree_import parses a caller's host blob: every size, count and
    # index in it is checked against the bytes present before the first CUDA
    # call, so truncated or corrupt blobs (including counts chosen to wrap the
    # size arithmetic) are rejected with FMT_EINVAL and never read past the
    # buffer.  A valid blob passes every host check: on a machine without a
    # GPU it then fails at the device (FMT_ECUDA).
    import struct
    torch = pytest.importorskip("torch")
    T, blob = _oracle_blob()
    K, nm = T.n_nodes, T.nmono
    assert K > 9 and int(T.depth.max()) == 2
    lib = F.load()

    def imp(b):
        h = ctypes.c_void_p()
        buf = (ctypes.c_char * max(len(b), 1)).from_buffer_copy(b if b else b"\0")
        st = lib.fmt_tree_import(buf, len(b), None, ctypes.byref(h))
        if h.value:
            lib.fmt_tree_free(h)
        return st

    assert imp(blob) == (F.FMT_OK if torch.cuda.is_available() else F.FMT_ECUDA)
    for n in range(len(blob)):
        assert imp(blob[:n]) == F.FMT_EINVAL, n

    hs = ctypes.sizeof(F.fmt_export_header)

    def header(**kw):
        h = F.fmt_export_header.from_buffer_copy(blob)
        for k, v in kw.items():
            if k == "level_nodes":
                for i in range(len(h.level_nodes)):
                    h.level_nodes[i] = v[i] if i < len(v) else 0
            else:
                setattr(h, k, v)
        return bytes(h) + blob[hs:]

    lv = [int(c) for c in np.bincount(T.depth)]
    bad_headers = [dict(magic=0), dict(version=1), dict(degree=15), dict(nmono=nm + 1), dict(n_levels=0),
                   dict(n_levels=23), dict(n_nodes=0), dict(n_problems=0), dict(n_problems=2 ** 31 - 1),
                   dict(n_levels=2, n_nodes=2 ** 62, level_nodes=[1, 2 ** 62 - 1]),  # wraps K * bytes per node
                   dict(n_levels=2, n_nodes=2 ** 57, level_nodes=[1, 2 ** 57 - 1]),
                   dict(n_nodes=K + 1, level_nodes=lv[:-1] + [lv[-1] + 1]),
                   dict(level_nodes=[0] + lv[1:]),
                   dict(level_nodes=[lv[0] + 5, lv[1] - 5] + lv[2:]),
                   dict(n_levels=2, level_nodes=[lv[0], lv[1] + lv[2]])]
    for kw in bad_headers:
        assert imp(header(**kw)) == F.FMT_EINVAL, kw

    def patch(off, fmt, value):
        b = bytearray(blob)
        struct.pack_into(fmt, b, hs + off, value)
        return bytes(b)

    prefix0 = struct.unpack_from("<Q", blob, hs + 8 * lv[0])[0]  # first node of level 1
    depth_at, nprob_at = 24 * K, 24 * K + 16 * K
    prob_at = K * (176 + 8 * nm)
    bad_bodies = [patch(8 * (lv[0] + 1), "<Q", prefix0),        # level 1 not strictly increasing
                  patch(depth_at + 4 * 1, "<i", 0),             # a level-1 node labelled depth 0
                  patch(nprob_at, "<i", 1),                     # node of problem 1 in a 1-problem blob
                  patch(nprob_at + 4 * (K - 1), "<i", -1),
                  patch(prob_at, "<i", T.degree + 1),           # problem degree above the blob's
                  patch(prob_at + 8 + 8 + 8 + 24, "<d", -1.0),  # problem side
                  patch(prob_at + 8 + 8 + 8 + 24, "<d", float("nan")),
                  patch(prob_at + 8 + 8 + 8, "<d", float("inf"))]   # problem lo
    for i, b in enumerate(bad_bodies):
        assert imp(b) == F.FMT_EINVAL, i


def test_shared_memory_limits_go_through_the_never_lowering_helper():
    # The dynamic shared-memory limit belongs to a kernel, not to one launch:
    # a launcher that set it directly to its own need could lower it under
    # another thread's launch of the same kernel.  Only fmt_smem_at_least,
    # which raises the limit and never lowers it, calls the runtime for it.
    csrc = os.path.join(ROOT, "paper_1511_01353_gb300", "csrc")
    calls = []
    for fn in sorted(os.listdir(csrc)):
        if fn.endswith((".cu", ".cuh")):
            src = open(os.path.join(csrc, fn)).read()
            for m in re.finditer(r"cudaFuncSetAttribute\s*\(", src):
                calls.append((fn, src.count("\n", 0, m.start())))
    assert len(calls) == 1, calls
    fn, line = calls[0]
    before = open(os.path.join(csrc, fn)).read().splitlines()[max(0, line - 12):line]
    assert any("fmt_smem_at_least(" in s for s in before), (fn, line)
