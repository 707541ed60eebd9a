"""Forests: many independent problems fitted together (oct_build_batch).

Each problem of the forest is checked against the oracle fitted on that
problem alone (its own degree, box and tau): bit-exact structure; residuals,
node polynomials and evaluated targets within 1e-10 * max|f| of that problem.
The forest mixes degrees 1..8, boxes and clustered clouds, so some nodes
have ill-conditioned bases (their points fill only part of their box): there
two correct FP64 solvers agree on the polynomial at the data but may differ
by cond * eps elsewhere, so polynomials and targets are compared at (or
next to) the data points.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1511_01353_gb300 import workloads as W
from tests import treecmp as TC
from tests.test_gpu_parity import dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _forest_case(seed=3):
    rng = np.random.default_rng(seed)
    specs = [  # (n, degree, lo, side, clustered)
        (3000, 4, (0.0, 0.0, 0.0), 1.0, False),
        (12, 4, (0.0, 0.0, 0.0), 1.0, False),       # fewer points than monomials: degree clamp
        (2500, 2, (-1.0, 2.0, 0.5), 3.0, False),
        (1, 3, (0.0, 0.0, 0.0), 1.0, False),        # single point
        (6000, 6, (0.0, 0.0, 0.0), 1.0, True),
        (900, 1, (5.0, 5.0, 5.0), 0.25, False),
        (4096, 8, (0.0, 0.0, 0.0), 1.0, True),
        (700, 5, (0.0, 0.0, 0.0), 2.0, False),
    ]
    xs, ys, zs, fs, boxes, degs = [], [], [], [], [], []
    for n, p, lo, side, clu in specs:
        if clu:
            # a cluster wide enough that the root fit stays well conditioned:
            # a tight cluster in a large box makes the root basis nearly
            # dependent (cond ~ 1e6..1e9), and two correct FP64 solvers then
            # differ by cond * eps away from the data
            c = np.array(lo) + side * rng.uniform(0.4, 0.6, 3)
            pts = np.clip(c + 0.25 * side * rng.normal(size=(n, 3)), np.array(lo), np.array(lo) + side * (1 - 1e-12))
        else:
            pts = np.array(lo) + side * rng.uniform(0, 1, (n, 3))
        x, y, z = pts[:, 0].copy(), pts[:, 1].copy(), pts[:, 2].copy()
        u = (x - lo[0]) / side
        v = (y - lo[1]) / side
        w = (z - lo[2]) / side
        xs.append(x); ys.append(y); zs.append(z); fs.append(W.franke_bj(u, v, w) * (1 + p))
        boxes.append(list(lo) + [side]); degs.append(p)
    offsets = np.concatenate([[0], np.cumsum([s[0] for s in specs])]).astype(np.int64)
    return specs, offsets, np.array(degs, np.int32), np.array(boxes), xs, ys, zs, fs


def test_forest_matches_oracle_per_problem():
    from paper_1511_01353_gb300 import fmt as F
    specs, offsets, degs, boxes, xs, ys, zs, fs = _forest_case()
    D, mp, tol_rel = 4, 16, 1e-6
    params = F.make_params(4, D, mp, tol_rel)
    cat = lambda a: dev(np.concatenate(a))
    tree = F.oct_build_batch(params, offsets, cat(xs), cat(ys), cat(zs), cat(fs), degrees=degs, boxes=boxes)
    F.fit_all(tree)
    ex = F.parse_export(F.fmt_tree_export(tree))
    assert ex.header["n_problems"] == len(specs)
    allxyz = (np.concatenate(xs), np.concatenate(ys), np.concatenate(zs))
    rng = np.random.default_rng(11)
    tq, tp = [], []
    for i, (n, p, lo, side, _) in enumerate(specs):
        T = O.fit(xs[i], ys[i], zs[i], fs[i], p, D, mp, tol_rel, lo=lo, side=side)
        tol = 1e-10 * max(T.maxabs, 1e-300)
        assert ex.problems["tau"][i] == T.tau and ex.problems["degree"][i] == p
        TC.compare_trees(T, ex, tol, problem=i, data_xyz=allxyz)
        sl = slice(offsets[i], offsets[i + 1])
        assert np.max(np.abs(ex.resid[sl] - T.resid)) <= tol
        pick = rng.integers(0, n, 200)  # targets next to data points (jitter 1e-6 of the box)
        q = np.stack([xs[i][pick], ys[i][pick], zs[i][pick]], axis=1) + 1e-6 * side * rng.normal(size=(200, 3))
        tq.append(q)
        tp.append(np.full(200, i, np.int32))
    q = np.concatenate(tq)
    prob = np.concatenate(tp)
    out = torch.empty(q.shape[0], dtype=torch.float64, device="cuda")
    nout = F.evaluate_batch(tree, torch.from_numpy(prob).cuda(), dev(q[:, 0]), dev(q[:, 1]), dev(q[:, 2]), out,
                            count_outside=True)
    got = out.cpu().numpy()
    n_out_ref = 0
    for i, (n, p, lo, side, _) in enumerate(specs):
        T = O.fit(xs[i], ys[i], zs[i], fs[i], p, D, mp, tol_rel, lo=lo, side=side)
        sel = prob == i
        ref, no = T.evaluate(q[sel, 0], q[sel, 1], q[sel, 2])
        n_out_ref += no
        assert np.max(np.abs(got[sel] - ref)) <= 1e-10 * max(T.maxabs, 1e-300)
    assert nout == n_out_ref


def test_single_problem_batch_equals_oct_build():
    from paper_1511_01353_gb300 import fmt as F
    w = W.scale(n=20000, n_targets=10)
    p = F.make_params(w.degree, w.max_depth, w.min_pts, w.tol_rel)
    a = F.parse_export(F.fmt_tree_export(F.fit(p, dev(w.x), dev(w.y), dev(w.z), dev(w.f))))
    t = F.oct_build_batch(p, np.array([0, w.n]), dev(w.x), dev(w.y), dev(w.z), dev(w.f))
    b = F.parse_export(F.fmt_tree_export(F.fit_all(t)))
    assert np.array_equal(a.prefix, b.prefix) and np.array_equal(a.coef, b.coef)
    assert np.array_equal(a.resid, b.resid)


def test_batch_argument_errors():
    from paper_1511_01353_gb300 import fmt as F
    x = dev(np.random.default_rng(0).uniform(0, 1, 100))
    p = F.make_params(3, 3, 10, 1e-4)
    with pytest.raises(F.FmtError):
        F.oct_build_batch(p, np.array([0, 50, 50, 100]), x, x, x, x)   # empty problem
    with pytest.raises(F.FmtError):
        F.oct_build_batch(p, np.array([0, 100]), x, x, x, x, degrees=np.array([15], np.int32))
    pdeep = F.make_params(3, 21, 10, 1e-4)
    with pytest.raises(F.FmtError):                                   # no key bits left for 3 problems
        F.oct_build_batch(pdeep, np.array([0, 30, 60, 100]), x, x, x, x)
    t = F.oct_build_batch(p, np.array([0, 40, 100]), x, x, x, x)
    F.fit_all(t)
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FmtError):
        F.evaluate_batch(t, torch.tensor([0, 1, 7], dtype=torch.int32, device="cuda"), x[:3], x[:3], x[:3], out,
                         count_outside=True)


def test_batched_recipe_against_oracle():
    """The batched recipe (degrees 4..10, uniform and clustered clouds,
    Franke and Gaussian-sum values, tol 1e-6) at 20 problems: every problem's
    tree against the oracle at its data points and targets."""
    from paper_1511_01353_gb300 import fmt as F
    b = W.batch(n_problems=20, n_max=6000, targets_per_problem=300, seed=W.SEED_BASE + 77)
    params = F.make_params(4, b.max_depth, b.min_pts, b.tol_rel)
    tree = F.oct_build_batch(params, b.offsets, dev(b.x), dev(b.y), dev(b.z), dev(b.f), degrees=b.degrees,
                             boxes=b.boxes)
    F.fit_all(tree)
    ex = F.parse_export(F.fmt_tree_export(tree))
    out = torch.empty(b.xq.shape[0], dtype=torch.float64, device="cuda")
    F.evaluate_batch(tree, torch.from_numpy(b.tprob).cuda(), dev(b.xq), dev(b.yq), dev(b.zq), out)
    got = out.cpu().numpy()
    allxyz = (b.x, b.y, b.z)
    worst = []
    for i in range(b.n_problems):
        s, e = int(b.offsets[i]), int(b.offsets[i + 1])
        T = O.fit(b.x[s:e], b.y[s:e], b.z[s:e], b.f[s:e], int(b.degrees[i]), b.max_depth, b.min_pts, b.tol_rel)
        tol = 1e-10 * T.maxabs
        TC.compare_trees(T, ex, tol, problem=i, data_xyz=allxyz)
        assert np.max(np.abs(ex.resid[s:e] - T.resid)) <= tol
        ts, te = int(b.toff[i]), int(b.toff[i + 1])
        ref, _ = T.evaluate(b.xq[ts:te], b.yq[ts:te], b.zq[ts:te])
        # Targets are fresh samples of the problem's cloud: in the tails of a
        # clustered cloud they can fall where an ill-conditioned node has no
        # data, and there two correct solvers differ by cond * eps; the
        # 1e-10 bar is held at the data points above.
        worst.append(float(np.max(np.abs(got[ts:te] - ref)) / T.maxabs))
    assert max(worst) <= 1e-6, worst
