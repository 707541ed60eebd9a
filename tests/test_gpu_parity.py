"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bar (from the method's statement of the FP64 path): Morton codes, the sort
permutation and the octree structure bit-exact; residuals, node polynomials
and interpolant values within 1e-10 * max|f|.
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


def gpu_fit(x, y, z, f, degree, max_depth, min_pts, tol_rel, chunk_rows=0, lo=(0.0, 0.0, 0.0), side=1.0):
    from paper_1511_01353_gb300 import fmt as F
    p = F.make_params(degree, max_depth, min_pts, tol_rel, lo=lo, side=side, chunk_rows=chunk_rows)
    tree = F.fit(p, dev(x), dev(y), dev(z), dev(f))
    ex = F.parse_export(F.fmt_tree_export(tree))
    return tree, ex


def gpu_eval(tree, xq, yq, zq):
    from paper_1511_01353_gb300 import fmt as F
    out = torch.empty(len(xq), dtype=torch.float64, device="cuda")
    nout = F.evaluate(tree, dev(xq), dev(yq), dev(zq), out, count_outside=True)
    torch.cuda.synchronize()
    return out.cpu().numpy(), nout


def check_case(x, y, z, f, degree, max_depth, min_pts, tol_rel, xq=None, yq=None, zq=None, chunk_rows=0,
               lo=(0.0, 0.0, 0.0), side=1.0):
    T = O.fit(x, y, z, f, degree, max_depth, min_pts, tol_rel, lo=lo, side=side)
    tree, ex = gpu_fit(x, y, z, f, degree, max_depth, min_pts, tol_rel, chunk_rows=chunk_rows, lo=lo, side=side)
    tol = REL_TOL * max(T.maxabs, 1e-300)
    assert ex.header["tau"] == T.tau
    assert ex.header["maxabs_f"] == T.maxabs
    # sorted Morton codes and permutation, bit-exact (independent numpy restatement)
    code = TC.morton_np(x, y, z, lo, side)
    sort_levels = min(max_depth + 1, 21)
    keys = code >> np.uint64(3 * (21 - sort_levels))
    perm = np.argsort(keys, kind="stable")
    assert np.array_equal(ex.perm, perm)
    assert np.array_equal(ex.code, code[perm])
    TC.compare_trees(T, ex, tol)
    assert np.max(np.abs(ex.resid - T.resid)) <= tol
    if xq is not None:
        a, na = gpu_eval(tree, xq, yq, zq)
        b, nb = T.evaluate(xq, yq, zq)
        assert na == nb
        assert np.max(np.abs(a - b)) <= tol
    return T, tree, ex


def test_small_workload():
    w = W.small()
    T, tree, ex = check_case(w.x, w.y, w.z, w.f, w.degree, w.max_depth, w.min_pts, w.tol_rel, w.xq, w.yq, w.zq)
    assert T.n_nodes == ex.prefix.shape[0] > 9


@pytest.mark.parametrize("chunk_rows", [0, 192, 512])
def test_scale_recipe_reduced(chunk_rows):
    # the 1e6-point clustered recipe at 3e4 points: several levels, TSQR over many chunks
    w = W.scale(n=30000, n_targets=20000)
    T, tree, ex = check_case(w.x, w.y, w.z, w.f, w.degree, w.max_depth, w.min_pts, w.tol_rel, w.xq, w.yq, w.zq,
                             chunk_rows=chunk_rows)
    assert T.depth.max() >= 2


def test_ragged_sizes_and_degrees():
    rng = np.random.default_rng(31)
    for n, p, D, mp in [(1, 3, 2, 1), (7, 2, 2, 1), (19, 4, 3, 1), (35, 4, 2, 1), (97, 2, 3, 10), (1000, 1, 4, 8),
                        (2049, 5, 3, 60), (3001, 6, 2, 90)]:
        x, y, z = (rng.uniform(0, 1, n) for _ in range(3))
        f = W.franke_paper(x, y, z)
        xq, yq, zq = (rng.uniform(0, 1, 333) for _ in range(3))
        check_case(x, y, z, f, p, D, mp, 1e-5, xq, yq, zq, chunk_rows=64 * (1 + n % 3))


def test_identity_and_polynomial_reproduction():
    rng = np.random.default_rng(5)
    n = 5000
    x, y, z = (rng.uniform(0, 1, n) for _ in range(3))
    xq, yq, zq = (rng.uniform(0, 1, 1000) for _ in range(3))
    T, tree, ex = check_case(x, y, z, np.ones(n), 6, 3, 84, 1e-9, xq, yq, zq)
    a, _ = gpu_eval(tree, xq, yq, zq)
    assert np.max(np.abs(a - 1.0)) <= 1e-12
    E = TC.exponents(3)
    cf = rng.normal(size=len(E))
    g = sum(cf[k] * x ** l * y ** m * z ** q for k, (l, m, q) in enumerate(E))
    gq = sum(cf[k] * xq ** l * yq ** m * zq ** q for k, (l, m, q) in enumerate(E))
    T, tree, ex = check_case(x, y, z, g, 3, 3, 20, 1e-8, xq, yq, zq)
    a, _ = gpu_eval(tree, xq, yq, zq)
    assert ex.prefix.shape[0] == 1
    assert np.max(np.abs(a - gq)) <= 1e-11 * np.max(np.abs(g))


def test_degenerate_point_sets():
    rng = np.random.default_rng(9)
    # duplicates: 20 distinct points repeated 10 times; 35 monomials of degree
    # <= 4 on 20 sites -> rank 20, 15 columns dropped on both sides
    b = rng.uniform(0, 1, (20, 3))
    pts = np.repeat(b, 10, axis=0)
    x, y, z = pts[:, 0].copy(), pts[:, 1].copy(), pts[:, 2].copy()
    f = W.franke_bj(x, y, z)
    T = O.fit(x, y, z, f, 4, 2, 35, 1e-6)
    tree, ex = gpu_fit(x, y, z, f, 4, 2, 35, 1e-6)
    assert ex.flags[0] & 2 and T.flags[0] & 2
    assert np.array_equal(ex.coef[0] == 0.0, T.coef[0] == 0.0)  # same columns dropped
    assert np.count_nonzero(T.coef[0]) == 20
    tol = REL_TOL * T.maxabs * 1e3  # square 20x20 interpolation, conditioned worse than the LS cases
    assert np.max(np.abs(ex.resid - T.resid)) <= tol
    a, _ = gpu_eval(tree, b[:, 0], b[:, 1], b[:, 2])
    assert np.max(np.abs(a - W.franke_bj(b[:, 0], b[:, 1], b[:, 2]))) <= tol
    # coplanar points
    n = 900
    x, y = rng.uniform(0, 1, n), rng.uniform(0, 1, n)
    z = np.full(n, 0.3)
    check_case(x, y, z, 1 + x * y - y ** 2, 2, 2, 10, 1e-6)
    # every point in one octant, and points exactly on dyadic faces
    x, y, z = (rng.uniform(0.5, 1.0, 800) for _ in range(3))
    x[:100] = 0.5
    y[100:200] = 0.75
    z[200:260] = 1.0
    check_case(x, y, z, W.franke_bj(x, y, z), 2, 4, 10, 1e-4, x[:300], y[:300], z[:300])
    # zero function: tau = 0, nothing refines
    T, tree, ex = check_case(x, y, z, np.zeros_like(x), 2, 3, 10, 1e-3)
    assert ex.prefix.shape[0] == 1 and np.all(ex.coef == 0)


def test_root_box_and_outside_targets():
    rng = np.random.default_rng(2)
    n = 3000
    lo, side = (-1.0, -2.0, 0.5), 4.0
    x, y, z = (lo[a] + side * rng.uniform(0, 1, n) for a in range(3))
    f = np.sin(x) * np.cos(y) + z
    xq = np.concatenate([rng.uniform(-2, 4, 400), [lo[0], lo[0] + side]])
    yq = np.concatenate([rng.uniform(-3, 3, 400), [lo[1], lo[1] + side]])
    zq = np.concatenate([rng.uniform(0, 5, 400), [lo[2], lo[2] + side]])
    check_case(x, y, z, f, 3, 3, 20, 1e-5, xq, yq, zq, lo=lo, side=side)


def test_targets_that_are_not_numbers_or_infinite():
    # NaN and infinite targets lie outside every cube: counted in n_outside,
    # and the targets beside them evaluate as they do alone
    rng = np.random.default_rng(4)
    x, y, z = rng.uniform(0, 1, (3, 2000))
    f = np.cos(2 * x) * y + z
    tree, ex = gpu_fit(x, y, z, f, 3, 3, 20, 1e-5)
    xq, yq, zq = rng.uniform(0, 1, (3, 300))
    base, n0 = gpu_eval(tree, xq, yq, zq)
    assert n0 == 0
    bad = [3, 50, 51, 199, 250]
    xb, yb, zb = xq.copy(), yq.copy(), zq.copy()
    xb[3], yb[50], zb[51], xb[199], yb[250] = np.nan, np.inf, -np.inf, -np.nan, np.nan
    a, na = gpu_eval(tree, xb, yb, zb)
    assert na == len(bad)
    keep = np.setdiff1d(np.arange(300), bad)
    assert np.array_equal(a[keep], base[keep])


def test_evaluate_imported_oracle_tree():
    """Evaluation alone: upload the oracle's tree through fmt_tree_import."""
    from paper_1511_01353_gb300 import fmt as F
    w = W.scale(n=20000, n_targets=30000)
    T = O.fit(w.x, w.y, w.z, w.f, w.degree, w.max_depth, w.min_pts, w.tol_rel)
    pref = (TC.spread3(T.ixyz[:, 0]) | (TC.spread3(T.ixyz[:, 1]) << np.uint64(1)) |
            (TC.spread3(T.ixyz[:, 2]) << np.uint64(2)))
    order = np.lexsort((pref, T.depth))
    hdr = dict(degree=T.degree, nmono=T.nmono, max_depth=T.max_depth, min_pts=T.min_pts, tol_rel=T.tol_rel,
               tau=T.tau, maxabs_f=T.maxabs, lo=T.lo, side=T.side, n_points=w.n)
    blob = F.build_export(hdr, pref[order], T.depth[order], T.flags[order], T.deg_used[order], T.child_E[order],
                          T.child_n[order], T.coef[order])
    tree = F.fmt_tree_import(blob)
    a, na = gpu_eval(tree, w.xq, w.yq, w.zq)
    b, nb = T.evaluate(w.xq, w.yq, w.zq)
    assert na == nb == 0
    assert np.max(np.abs(a - b)) <= REL_TOL * T.maxabs
    ex = F.parse_export(F.fmt_tree_export(tree))
    assert np.array_equal(ex.coef, T.coef[order])
    with pytest.raises(F.FmtError):
        F.fit_level(tree, 0)


def test_call_order_and_input_errors():
    from paper_1511_01353_gb300 import fmt as F
    rng = np.random.default_rng(1)
    x, y, z = (rng.uniform(0, 1, 500) for _ in range(3))
    p = F.make_params(2, 3, 10, 1e-4)
    tree = F.oct_build(p, dev(x), dev(y), dev(z), dev(x * y))
    with pytest.raises(F.FmtError):
        F.refine(tree, 0)           # refine before fit
    with pytest.raises(F.FmtError):
        F.fit_level(tree, 1)        # wrong depth
    out = torch.empty(10, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FmtError):
        F.evaluate(tree, dev(x[:10]), dev(y[:10]), dev(z[:10]), out)  # nothing fitted yet
    F.fit_level(tree, 0)
    with pytest.raises(F.FmtError):
        F.fit_level(tree, 0)        # twice
    F.refine(tree, 0)
    assert F.evaluate(tree, dev(x[:0]), dev(y[:0]), dev(z[:0]), out[:0], count_outside=True) == 0
    bad = x.copy()
    bad[17] = np.nan
    with pytest.raises(F.FmtError) as e:
        F.oct_build(p, dev(bad), dev(y), dev(z), dev(x))
    assert e.value.status == F.FMT_EINVAL
    badf = x.copy()
    badf[3] = np.inf
    with pytest.raises(F.FmtError):
        F.oct_build(p, dev(x), dev(y), dev(z), dev(badf))


def test_stats_and_determinism():
    from paper_1511_01353_gb300 import fmt as F
    w = W.scale(n=20000, n_targets=100)
    t1, e1 = gpu_fit(w.x, w.y, w.z, w.f, w.degree, w.max_depth, w.min_pts, w.tol_rel)
    t2, e2 = gpu_fit(w.x, w.y, w.z, w.f, w.degree, w.max_depth, w.min_pts, w.tol_rel)
    assert np.array_equal(e1.coef, e2.coef) and np.array_equal(e1.resid, e2.resid)  # run to run, bitwise
    s = F.fmt_tree_stats(t1)
    assert s.n_levels == s.n_fitted == len([d for d in range(22) if s.nodes[d] > 0])
    assert s.nodes[0] == 1 and s.points[0] == w.n
    assert sum(s.nodes[d] for d in range(22)) == e1.prefix.shape[0]


@pytest.mark.parametrize("p,n,D", [(10, 3000, 1), (12, 5000, 1), (14, 7000, 1)])
def test_high_degrees(p, n, D):
    # the degrees of the paper's unscoped runs (nmono 286, 455, 680); the
    # triangles no longer fit in shared memory, so the merges take the
    # general path.  Monomials of degree 14 on [-1,1]^3 scaled by 1/(l!m!n!)
    # make kappa ~ 1e13, so node polynomials are compared at the node's own
    # data points, where the least-squares fit is determined.
    rng = np.random.default_rng(100 + p)
    x, y, z = (rng.uniform(0, 1, n) for _ in range(3))
    f = W.franke_paper(x, y, z)
    T = O.fit(x, y, z, f, p, D, 1, 1e-12)
    tree, ex = gpu_fit(x, y, z, f, p, D, 1, 1e-12, chunk_rows=1024)
    tol = REL_TOL * T.maxabs
    TC.compare_trees(T, ex, tol, data_xyz=(x, y, z))
    assert np.max(np.abs(ex.resid - T.resid)) <= tol
