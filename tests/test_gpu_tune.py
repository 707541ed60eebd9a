"""Launch configurations of the FP64 fit (fmt_tune_set / fmt_autotune) and
the CUDA-graph form of fit_level (FMT_OPT_GRAPH) on the GPU.

A configuration changes the rows per shared-memory block, the warps per
tile-QR CTA, the row chunks of a node and the merge kernel, i.e. the order of
the floating-point operations of the Householder QR, not the method: each one
meets the FP64 bar (1e-10 max|f|) against the oracle.  The graph form
replays the same kernels in the same order, so its results are bitwise
those of the stream form.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1511_01353_gb300 import workloads as W
from tests import treecmp as TC

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_TOL = 1e-10


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.fixture(scope="module")
def clustered():
    # the clustered recipe at 2.4e4 points, degree 8: several levels, nodes
    # of very different sizes, large nodes split into many chunks
    w = W.scale(n=24000, n_targets=5000)
    T = O.fit(w.x, w.y, w.z, w.f, 8, 4, 128, 1e-6)
    return w, T


def fit_export(w, graph=False, precision=0):
    from paper_1511_01353_gb300 import fmt as F
    p = F.make_params(8, 4, 128, 1e-6, precision=precision, graph=graph)
    tree = F.fit(p, dev(w.x), dev(w.y), dev(w.z), dev(w.f))
    return tree, F.parse_export(F.fmt_tree_export(tree))


def eval_tree(tree, w):
    from paper_1511_01353_gb300 import fmt as F
    out = torch.empty(len(w.xq), dtype=torch.float64, device="cuda")
    F.evaluate(tree, dev(w.xq), dev(w.yq), dev(w.zq), out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


CONFIGS = [(rows, warps, cf, merge) for rows in (16, 32, 48, 64, 128) for warps in (4, 8)
           for cf, merge in ((1, 0), (16, 1))]


@pytest.mark.parametrize("rows,warps,chunk_factor,merge", CONFIGS)
def test_every_configuration_meets_the_fp64_bar(clustered, rows, warps, chunk_factor, merge):
    from paper_1511_01353_gb300 import fmt as F
    w, T = clustered
    F.fmt_tune_set(dict(degree=8, rows=rows, warps=warps, chunk_factor=chunk_factor, merge=merge))
    try:
        tree, ex = fit_export(w)
        st = F.fmt_tree_stats(tree)
        tol = REL_TOL * T.maxabs
        TC.compare_trees(T, ex, tol)
        assert np.max(np.abs(ex.resid - T.resid)) <= tol
        b, _ = T.evaluate(w.xq, w.yq, w.zq)
        assert np.max(np.abs(eval_tree(tree, w) - b)) <= tol
        if chunk_factor == 1:  # small chunks: the root is split into several items that are merged
            assert int(st.items[0]) > 1
    finally:
        F.fmt_tune_set(dict(degree=8, source=0))


def test_autotune_installs_a_measured_entry(clustered):
    from paper_1511_01353_gb300 import fmt as F
    w, T = clustered
    try:
        e = F.fmt_autotune(8, sample_points=1 << 17)
        assert e["source"] == 1 and e["degree"] == 8 and e["sample_points"] == 1 << 17
        assert e["trials"] >= 8
        assert 0.0 < e["ms"] <= e["ms_builtin"]
        assert F.fmt_tune_get(8) == e
        tree, ex = fit_export(w)
        TC.compare_trees(T, ex, REL_TOL * T.maxabs)
        assert np.max(np.abs(ex.resid - T.resid)) <= REL_TOL * T.maxabs
    finally:
        F.fmt_tune_set(dict(degree=8, source=0))


def test_autotune_rejects_bad_arguments():
    from paper_1511_01353_gb300 import fmt as F
    for deg, n in ((15, 0), (-1, 0), (4, -5)):
        with pytest.raises(F.FmtError):
            F.fmt_autotune(deg, sample_points=n)


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_form_is_bitwise_the_stream_form(clustered, precision):
    from paper_1511_01353_gb300 import fmt as F
    w, _ = clustered
    _, ref = fit_export(w, graph=False, precision=precision)
    F.fmt_profile_enable(True)
    _, g1 = fit_export(w, graph=True, precision=precision)  # instantiates (or updates) one graph per level
    _, g2 = fit_export(w, graph=True, precision=precision)  # same launch structure: updated in place
    prof = F.fmt_profile_read()
    F.fmt_profile_enable(False)
    for g in (g1, g2):
        assert np.array_equal(g.coef, ref.coef)
        assert np.array_equal(g.resid, ref.resid)
        assert np.array_equal(g.flags, ref.flags)
    levels = int(ref.header["n_levels"])
    gl = prof["graph_launch"]
    assert gl["launches"] == 2 * levels
    assert gl["units"] >= levels  # the second fit reused every level's executable graph
    assert prof["tile_qr"]["ms"] > 0.0  # event timing works inside graphs


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_form_of_a_forest_of_several_degrees(precision):
    # a forest of degrees 4..10: the tile QR of a level forks one launch per
    # degree onto side streams; captured in a graph, the fork and join are
    # part of the graph, and the results are bitwise those of the stream form
    from paper_1511_01353_gb300 import fmt as F
    b = W.batch(n_problems=20, n_min=300, n_max=6000)

    def run(graph):
        p = F.make_params(4, b.max_depth, b.min_pts, b.tol_rel, precision=precision, graph=graph)
        tree = F.oct_build_batch(p, b.offsets, dev(b.x), dev(b.y), dev(b.z), dev(b.f), degrees=b.degrees,
                                 boxes=b.boxes)
        F.fit_all(tree)
        return F.parse_export(F.fmt_tree_export(tree))

    ref, g = run(False), run(True)
    assert len(set(int(d) for d in b.degrees)) > 2
    assert np.array_equal(g.coef, ref.coef)
    assert np.array_equal(g.resid, ref.resid)
    assert np.array_equal(g.flags, ref.flags)


def test_forest_tuner_keeps_the_fp64_bar():
    # The forest autotuner times the whole level loop of a mixed-degree forest
    # under candidate tables and installs the winners; whatever it picks, the
    # fit of every problem meets the FP64 bar against the oracle.
    from paper_1511_01353_gb300 import fmt as F
    b = W.batch(n_problems=16, n_min=300, n_max=6000, deg_min=3, deg_max=7)
    p = F.make_params(3, b.max_depth, b.min_pts, b.tol_rel)
    saved = {d: F.fmt_tune_get(d) for d in range(F.FMT_MAX_DEGREE + 1)}
    try:
        rep = F.fmt_autotune_forest(p, b.offsets, dev(b.x), dev(b.y), dev(b.z), dev(b.f), degrees=b.degrees,
                                    boxes=b.boxes)
        assert rep["trials"] >= 2 and rep["ms_start"] > 0.0 and rep["ms_best"] <= rep["ms_start"]
        tree = F.fit_all(F.oct_build_batch(p, b.offsets, dev(b.x), dev(b.y), dev(b.z), dev(b.f),
                                           degrees=b.degrees, boxes=b.boxes))
        ex = F.parse_export(F.fmt_tree_export(tree))
        tree.close()
        for i in range(b.n_problems):
            s, e = int(b.offsets[i]), int(b.offsets[i + 1])
            T = O.fit(b.x[s:e], b.y[s:e], b.z[s:e], b.f[s:e], int(b.degrees[i]), b.max_depth, b.min_pts, b.tol_rel)
            assert np.max(np.abs(ex.resid[s:e] - T.resid)) <= REL_TOL * T.maxabs
    finally:
        for d, e in saved.items():
            F.fmt_tune_set(dict(e, source=0) if e["source"] == 0 else e)
