"""Mixed-precision fit (FMT_MIXED) against the FP64 oracle.

The mixed path computes each node's least-squares fit (Alg. 2) from a Gram
matrix formed on the tensor cores (split-BF16 digit tiles, FP32 accumulation,
FP64 promotion), an FP64 Cholesky factor and FP64 refinement sweeps.  Nodes
that tier cannot fit (ill-conditioned, not converged, degree above 9) go to
its FP64 normal-equations tier (FP64 Gram, Cholesky, corrected semi-normal
sweeps); what neither fits (rank-deficient, clamped root), and the nearly
square nodes of a level with few of them, go to the FP64 Householder path
and then meet the FP64 bar of 1e-10.  The stated bar of
the mixed path is an interpolant within 1e-6 * max|f| of the FP64 oracle.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1511_01353_gb300 import workloads as W
from tests import treecmp as TC

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-6
FP64_TOL = 1e-10


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def mixed_fit(x, y, z, f, degree, max_depth, min_pts, tol_rel, sweeps=0, chunk_rows=0, lo=(0.0, 0.0, 0.0),
              side=1.0):
    from paper_1511_01353_gb300 import fmt as F
    p = F.make_params(degree, max_depth, min_pts, tol_rel, lo=lo, side=side, chunk_rows=chunk_rows,
                      precision=F.FMT_MIXED, sweeps=sweeps)
    tree = F.fit(p, dev(x), dev(y), dev(z), dev(f))
    return tree, F.parse_export(F.fmt_tree_export(tree)), F.fmt_tree_stats(tree)


def gpu_eval(tree, xq, yq, zq):
    from paper_1511_01353_gb300 import fmt as F
    out = torch.empty(len(xq), dtype=torch.float64, device="cuda")
    F.evaluate(tree, dev(xq), dev(yq), dev(zq), out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def mixed_points(st):
    return sum(int(st.mixed_points[d]) for d in range(st.n_levels))


def test_precision_form_of_the_small_workload():
    # 4096 uniform points, p = 8, depth 7, min 64, tol 1e-4 (the small workload at degree 8)
    w = W.small()
    T = O.fit(w.x, w.y, w.z, w.f, 8, 7, 64, 1e-4)
    tree, ex, st = mixed_fit(w.x, w.y, w.z, w.f, 8, 7, 64, 1e-4)
    tol = MIXED_TOL * T.maxabs
    assert int(st.mixed[0]) == 1  # the root went through the tensor-core path
    assert mixed_points(st) >= 0.9 * sum(int(st.points[d]) for d in range(st.n_levels))
    TC.compare_trees(T, ex, tol, data_xyz=(w.x, w.y, w.z))
    assert np.max(np.abs(ex.resid - T.resid)) <= tol
    a = gpu_eval(tree, w.xq, w.yq, w.zq)
    b, _ = T.evaluate(w.xq, w.yq, w.zq)
    err = np.max(np.abs(a - b)) / T.maxabs
    assert err <= MIXED_TOL, err


@pytest.mark.parametrize("chunk_rows", [0, 192])
def test_scale_recipe_reduced(chunk_rows):
    # the clustered 1e6-point recipe at 3e4 points; tau = 1e-8 max|f| makes a
    # few refinement decisions sensitive, so only the interpolant is compared
    w = W.scale(n=30000, n_targets=20000)
    T = O.fit(w.x, w.y, w.z, w.f, w.degree, w.max_depth, w.min_pts, w.tol_rel)
    tree, ex, st = mixed_fit(w.x, w.y, w.z, w.f, w.degree, w.max_depth, w.min_pts, w.tol_rel, chunk_rows=chunk_rows)
    assert mixed_points(st) >= 0.5 * sum(int(st.points[d]) for d in range(st.n_levels))
    a = gpu_eval(tree, w.xq, w.yq, w.zq)
    b, _ = T.evaluate(w.xq, w.yq, w.zq)
    err = np.max(np.abs(a - b)) / T.maxabs
    assert err <= MIXED_TOL, err


def test_polynomial_reproduction():
    # a degree-6 polynomial is reproduced by a single degree-6 node
    rng = np.random.default_rng(5)
    x, y, z = rng.uniform(0, 1, (3, 3000))
    c = rng.normal(size=(7, 7, 7))
    f = sum(c[a, b, g] * x ** a * y ** b * z ** g for a in range(7) for b in range(7 - a) for g in range(7 - a - b))
    tree, ex, st = mixed_fit(x, y, z, f, 6, 0, 1, 0.0)
    assert ex.flags[0] & 8
    assert np.max(np.abs(ex.resid)) <= 1e-8 * np.max(np.abs(f))


def test_resolution_of_identity():
    rng = np.random.default_rng(6)
    x, y, z = rng.uniform(0, 1, (3, 2000))
    tree, ex, st = mixed_fit(x, y, z, np.ones(2000), 8, 0, 1, 0.0)
    assert ex.flags[0] & 8
    xq, yq, zq = rng.uniform(0, 1, (3, 500))
    assert np.max(np.abs(gpu_eval(tree, xq, yq, zq) - 1.0)) <= 1e-9


def test_coplanar_points_fall_back_to_fp64():
    # z constant: the degree-4 basis is rank deficient, Cholesky breaks down
    rng = np.random.default_rng(7)
    x, y = rng.uniform(0, 1, (2, 800))
    z = np.full(800, 0.3)
    f = np.sin(3 * x) * np.cos(2 * y)
    T = O.fit(x, y, z, f, 4, 0, 1, 0.0)
    tree, ex, st = mixed_fit(x, y, z, f, 4, 0, 1, 0.0)
    assert not (ex.flags[0] & 8) and int(st.mixed[0]) == 0
    assert ex.flags[0] & 2 == T.flags[0] & 2
    assert np.max(np.abs(ex.resid - T.resid)) <= FP64_TOL * T.maxabs


@pytest.mark.parametrize("degree", [10, 12])
def test_degree_above_tensor_limit(degree):
    # degree 10: the FP64 normal-equations tier; degree 12: Householder
    rng = np.random.default_rng(8)
    x, y, z = rng.uniform(0, 1, (3, 3000))
    f = np.exp(-((x - 0.4) ** 2 + (y - 0.6) ** 2 + z ** 2))
    T = O.fit(x, y, z, f, degree, 0, 1, 0.0)
    tree, ex, st = mixed_fit(x, y, z, f, degree, 0, 1, 0.0)
    err = np.max(np.abs(ex.resid - T.resid)) / T.maxabs
    if degree <= 10:
        assert ex.flags[0] & 8 and ex.flags[0] & 64  # FMT_FLAG_MIXED | FMT_FLAG_MIXED_FP64
        assert err <= MIXED_TOL, err
    else:
        assert not (ex.flags[0] & 8)
        assert err <= FP64_TOL, err
    xq, yq, zq = rng.uniform(0, 1, (3, 2000))
    b, _ = T.evaluate(xq, yq, zq)
    assert np.max(np.abs(gpu_eval(tree, xq, yq, zq) - b)) / T.maxabs <= MIXED_TOL


@pytest.mark.parametrize("degree,n", [(4, 40), (6, 110), (8, 200)])
def test_nearly_square_nodes_take_householder(degree, n):
    # fewer than 1.5 m points (m = nmono + 1), more than nmono: the node skips
    # both normal-equations tiers, is refitted by Householder from the start
    # of its level and meets the FP64 bar
    rng = np.random.default_rng(10 + degree)
    x, y, z = rng.uniform(0, 1, (3, n))
    f = np.sin(2 * x) + y * z - z
    from paper_1511_01353_gb300 import fmt as F
    m = F.fmt_nmono(degree) + 1
    assert m - 1 <= n < 1.5 * m
    T = O.fit(x, y, z, f, degree, 0, 1, 0.0)
    tree, ex, st = mixed_fit(x, y, z, f, degree, 0, 1, 0.0)
    assert not (ex.flags[0] & 8) and int(st.mixed[0]) == 0
    assert np.max(np.abs(ex.resid - T.resid)) <= FP64_TOL * T.maxabs
    # the interpolant at the data points is f - r
    assert np.max(np.abs(gpu_eval(tree, x, y, z) - (f - T.resid))) <= FP64_TOL * T.maxabs


def test_clustered_nodes_across_the_tiers():
    # three Gaussian clusters in one root, narrower and narrower: the degree-9
    # basis grows ill-conditioned on the data, past the tensor-core Gram, then
    # past the FP64 normal equations (whose rounding-driven change over the
    # box is checked), then to numerical rank deficiency.  Each fit meets the
    # bar of the tier that took it (mixed 1e-6; Householder 1e-10).
    rng = np.random.default_rng(9)
    cs = np.array([[0.2, 0.3, 0.25], [0.7, 0.6, 0.8], [0.35, 0.8, 0.5]])
    seen = []
    for sigma in (0.25, 0.18, 0.12, 0.08, 0.05, 0.035, 0.025):
        pts = np.concatenate([c + sigma * rng.normal(size=(1500, 3)) for c in cs])
        x, y, z = np.clip(pts, 0.0, 0.999).T.copy()
        f = np.sin(4 * x) * np.cos(3 * y) + z * z
        T = O.fit(x, y, z, f, 9, 0, 1, 0.0)
        tree, ex, st = mixed_fit(x, y, z, f, 9, 0, 1, 0.0)
        fl = int(ex.flags[0])
        err = np.max(np.abs(ex.resid - T.resid)) / T.maxabs
        seen.append((sigma, fl, err))
        assert err <= (MIXED_TOL if fl & 8 else FP64_TOL), seen[-1]
    print("sigma, root flags, error:", seen)
    assert seen[0][1] & 8 and seen[-1][1] & 2  # the widest on the tensor cores, the narrowest rank-deficient


def test_sweeps_reduce_the_error():
    w = W.small()
    T = O.fit(w.x, w.y, w.z, w.f, 8, 0, 1, 0.0)
    errs = []
    for sw in (-1, 2, 3):
        tree, ex, st = mixed_fit(w.x, w.y, w.z, w.f, 8, 0, 1, 0.0, sweeps=sw)
        assert ex.flags[0] & 8, sw
        errs.append(np.max(np.abs(ex.resid - T.resid)) / T.maxabs)
    assert errs[2] <= errs[0]
    assert errs[2] <= 1e-8, errs


def test_forest_of_mixed_degrees():
    # Problems of degree 4..10 (degree 10 takes the FP64 tier) fitted in one
    # forest; the interpolant meets the mixed bar at each problem's data
    # points and at fresh targets of its cloud (a node is accepted only if
    # its polynomial has settled over its whole box, not only at its data).
    b = W.batch(n_problems=24, n_min=300, n_max=8000)
    from paper_1511_01353_gb300 import fmt as F
    p = F.make_params(4, b.max_depth, b.min_pts, b.tol_rel, precision=F.FMT_MIXED)
    tree = F.oct_build_batch(p, b.offsets, dev(b.x), dev(b.y), dev(b.z), dev(b.f), degrees=b.degrees,
                             boxes=b.boxes)
    F.fit_all(tree)
    ex = F.parse_export(F.fmt_tree_export(tree))
    out = torch.empty(len(b.xq), dtype=torch.float64, device="cuda")
    F.evaluate_batch(tree, torch.from_numpy(b.tprob).cuda(), dev(b.xq), dev(b.yq), dev(b.zq), out)
    a = out.cpu().numpy()
    st = F.fmt_tree_stats(tree)
    assert mixed_points(st) > 0
    assert np.any(ex.flags & 64)  # degree-10 problems (at least) took the FP64 tier
    report = []
    for i in range(b.n_problems):
        s, e = int(b.offsets[i]), int(b.offsets[i + 1])
        T = O.fit(b.x[s:e], b.y[s:e], b.z[s:e], b.f[s:e], int(b.degrees[i]), b.max_depth, b.min_pts, b.tol_rel)
        err_data = np.max(np.abs(ex.resid[s:e] - T.resid)) / T.maxabs
        ts, te = int(b.toff[i]), int(b.toff[i + 1])
        ref, _ = T.evaluate(b.xq[ts:te], b.yq[ts:te], b.zq[ts:te])
        err_t = np.max(np.abs(a[ts:te] - ref)) / T.maxabs
        report.append((i, int(b.degrees[i]), b.cloud[i], err_data, err_t))
        assert err_data <= MIXED_TOL, report[-1]
        assert err_t <= MIXED_TOL, report[-1]
    print("\n".join("problem %d p=%d %s: data %.2e targets %.2e" % r for r in report))


def test_run_to_run_bitwise():
    w = W.scale(n=20000, n_targets=10)
    _, ex1, _ = mixed_fit(w.x, w.y, w.z, w.f, w.degree, w.max_depth, w.min_pts, w.tol_rel)
    _, ex2, _ = mixed_fit(w.x, w.y, w.z, w.f, w.degree, w.max_depth, w.min_pts, w.tol_rel)
    assert np.array_equal(ex1.coef, ex2.coef)
    assert np.array_equal(ex1.resid, ex2.resid)
