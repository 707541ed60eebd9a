"""Parity at the benchmark's full size, in the configuration bench.py times.

1e6 points (half uniform, half in 8 Gaussian clusters), 3-D Franke values,
p = 8, max depth 7, min 128 points, tol 1e-8, automatic chunking.  The oracle
fits the whole tree (OpenMP over sibling subtrees; about a minute on 16
cores).  Checked: Morton codes and permutation and the tree structure
bit-exact; residuals and every node polynomial within 1e-10 * max|f|;
2e5 of the 1e7 evaluated targets against the oracle; the interpolant at the
1e6 data points equals f minus the final residual.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1511_01353_gb300 import workloads as W
from tests import treecmp as TC
from tests.test_gpu_parity import dev, gpu_eval, gpu_fit

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_scale_workload_full_size():
    from paper_1511_01353_gb300 import fmt as F
    w = W.scale()
    tree, ex = gpu_fit(w.x, w.y, w.z, w.f, w.degree, w.max_depth, w.min_pts, w.tol_rel)
    T = O.fit(w.x, w.y, w.z, w.f, w.degree, w.max_depth, w.min_pts, w.tol_rel, mode="omp")
    tol = 1e-10 * T.maxabs
    assert ex.header["tau"] == T.tau
    code = TC.morton_np(w.x, w.y, w.z)
    perm = np.argsort(code >> np.uint64(3 * (21 - min(w.max_depth + 1, 21))), kind="stable")
    assert np.array_equal(ex.perm, perm)
    assert np.array_equal(ex.code, code[perm])
    TC.compare_trees(T, ex, tol, n_poly_pts=4)
    assert np.max(np.abs(ex.resid - T.resid)) <= tol
    # all 1e7 targets on the GPU, a seeded sample against the oracle
    out = torch.empty(w.m, dtype=torch.float64, device="cuda")
    nout = F.evaluate(tree, dev(w.xq), dev(w.yq), dev(w.zq), out, count_outside=True)
    torch.cuda.synchronize()
    assert nout == 0
    sample = np.random.default_rng(1).choice(w.m, 200_000, replace=False)
    ref, _ = T.evaluate(w.xq[sample], w.yq[sample], w.zq[sample])
    assert np.max(np.abs(out.cpu().numpy()[sample] - ref)) <= tol
    # interpolant at the data points = f - final residual
    at_pts, _ = gpu_eval(tree, w.x, w.y, w.z)
    assert np.max(np.abs(at_pts - (w.f - ex.resid))) <= tol
