"""Exact metamorphic checks of the FP64 GPU path at the benchmark's full size
(1e6 clustered points, p = 8, depth 7, min 128 points, tol 1e-8).

Multiplying by a power of two commutes with IEEE rounding (no overflow or
underflow here), and the method is built from operations that are linear in
the values (the Householder steps act on the residual column linearly, the
back substitution, the residual update, E = sqrt(S/n) and tau = tol max|f|)
or that see only the points.  So:
  * fitting 4 f on the same points must give the same tree with every
    coefficient, residual and interpolated value multiplied by exactly 4;
  * doubling the points, the root cube's corner and its side must give the
    same Morton codes, tree, node frames (u = (x - c) s is unchanged) and so
    bitwise the same coefficients, residuals and values at doubled targets.
The oracle pins both on the CPU; these run the CUDA path, launch
configuration and chunking that bench.py times."""
import numpy as np
import pytest

from paper_1511_01353_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def run(w, x, y, z, f, xq, yq, zq, lo=(0.0, 0.0, 0.0), side=1.0):
    from paper_1511_01353_gb300 import fmt as F
    p = F.make_params(w.degree, w.max_depth, w.min_pts, w.tol_rel, lo=lo, side=side)
    tree = F.fit(p, dev(x), dev(y), dev(z), dev(f))
    out = torch.empty(xq.shape[0], dtype=torch.float64, device="cuda")
    F.evaluate(tree, dev(xq), dev(yq), dev(zq), out)
    torch.cuda.synchronize()
    ex = F.parse_export(F.fmt_tree_export(tree))
    tree.close()
    return ex, out.cpu().numpy()


@pytest.fixture(scope="module")
def scale():
    w = W.scale(n_targets=1_000_000)
    base = run(w, w.x, w.y, w.z, w.f, w.xq, w.yq, w.zq)
    return w, base


def test_four_f_scales_every_result_by_four(scale):
    w, (ex, out) = scale
    ex4, out4 = run(w, w.x, w.y, w.z, 4.0 * w.f, w.xq, w.yq, w.zq)
    assert np.array_equal(ex4.prefix, ex.prefix) and np.array_equal(ex4.count, ex.count)
    assert np.array_equal(ex4.flags, ex.flags)
    assert np.array_equal(ex4.coef, 4.0 * ex.coef)
    assert np.array_equal(ex4.resid, 4.0 * ex.resid)
    assert np.array_equal(ex4.child_E, 4.0 * ex.child_E)
    assert np.array_equal(out4, 4.0 * out)


def test_doubled_points_and_cube_change_nothing(scale):
    w, (ex, out) = scale
    ex2, out2 = run(w, 2.0 * w.x, 2.0 * w.y, 2.0 * w.z, w.f, 2.0 * w.xq, 2.0 * w.yq, 2.0 * w.zq,
                    lo=(0.0, 0.0, 0.0), side=2.0)
    assert np.array_equal(ex2.prefix, ex.prefix) and np.array_equal(ex2.count, ex.count)
    assert np.array_equal(ex2.flags, ex.flags)
    assert np.array_equal(ex2.coef, ex.coef)
    assert np.array_equal(ex2.resid, ex.resid)
    assert np.array_equal(out2, out)
