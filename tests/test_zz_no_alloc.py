"""The allocation-free entry point, fmt_fit_node_static.

Some callers cannot let a library allocate device memory: their device
memory belongs to another allocator or a fixed budget, or they must not risk
cudaMalloc's implicit device synchronisation and run-time out-of-memory
failures.  fmt_fit_node_static serves them: it fits one point set using a
static device array as its only scratch.  Here it is called through the C ABI
and its coefficients and residuals are checked against the tree path
(oct_build + fit_level at depth 0, which does the same fit with memory the
library allocates), on two calls in a row, within the tolerance of the other
parity tests (1e-10 * max|f|).

This file is named to be collected last.
"""
import numpy as np
import pytest

from paper_1511_01353_gb300 import workloads as W
from tests import treecmp as TC

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def tree_root_fit(x, y, z, f, degree):
    from paper_1511_01353_gb300 import fmt as F
    p = F.make_params(degree, 0, 1, 1e-6)
    tree = F.oct_build(p, dev(x), dev(y), dev(z), dev(f))
    F.fit_level(tree, 0)
    F.refine(tree, 0)
    ex = F.parse_export(F.fmt_tree_export(tree))
    tree.close()
    return ex.coef[0], ex.resid, int(ex.flags[0])


def test_static_fit_matches_tree_path_twice():
    from paper_1511_01353_gb300 import fmt as F
    rng = np.random.default_rng(77)
    # two calls in a row on one device: the second, smaller fit reuses the
    # scratch the first one filled
    for n, degree in [(6000, 8), (700, 5)]:
        x, y, z = (rng.uniform(0, 1, n) for _ in range(3))
        f = W.franke_bj(x, y, z)
        coef = torch.full((F.fmt_nmono(degree),), np.nan, dtype=torch.float64, device="cuda")
        r_out = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
        flags = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        F.fmt_fit_node_static(degree, dev(x), dev(y), dev(z), dev(f), coef, r_out, flags)
        torch.cuda.synchronize()
        c_tree, r_tree, fl_tree = tree_root_fit(x, y, z, f, degree)
        tol = 1e-10 * np.max(np.abs(f))
        assert int(flags.item()) == fl_tree == 0
        assert np.max(np.abs(r_out.cpu().numpy() - r_tree)) <= tol
        pts = rng.uniform(0, 1, (64, 3))
        key = (0, 0, 0, 0)
        a = TC.node_poly(coef.cpu().numpy(), degree, key, (0.0, 0.0, 0.0), 1.0, pts)
        b = TC.node_poly(c_tree, degree, key, (0.0, 0.0, 0.0), 1.0, pts)
        assert np.max(np.abs(a - b)) <= tol


def test_static_fit_allocates_nothing():
    """After one warm-up call (the symbol lookup and the module's first load),
    a call still succeeds while the library's next device allocation is set
    to fail, and the device's free memory is the same before and after it."""
    from paper_1511_01353_gb300 import fmt as F
    rng = np.random.default_rng(11)
    n, degree = 3000, 8
    x, y, z = (dev(rng.uniform(0, 1, n)) for _ in range(3))
    f = dev(W.franke_bj(x.cpu().numpy(), y.cpu().numpy(), z.cpu().numpy()))
    coef = torch.zeros(F.fmt_nmono(degree), dtype=torch.float64, device="cuda")
    r_out = torch.zeros(n, dtype=torch.float64, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    F.fmt_fit_node_static(degree, x, y, z, f, coef, r_out, flags)
    torch.cuda.synchronize()
    c0, r0 = coef.clone(), r_out.clone()
    free_before = torch.cuda.mem_get_info()[0]
    F.fmt_debug_fail_alloc(1)
    try:
        F.fmt_fit_node_static(degree, x, y, z, f, coef, r_out, flags)
        torch.cuda.synchronize()
    finally:
        F.fmt_debug_fail_alloc(0)
    free_after = torch.cuda.mem_get_info()[0]
    assert free_after == free_before
    # the same inputs give the same fit (the shared scratch is cleared before use)
    assert torch.equal(coef, c0) and torch.equal(r_out, r0)


def test_static_fit_degree_clamp_and_limit():
    from paper_1511_01353_gb300 import fmt as F
    rng = np.random.default_rng(5)
    n = 30  # fewer points than the 35 monomials of degree 4: degree lowered to 3
    x, y, z = (rng.uniform(0, 1, n) for _ in range(3))
    f = np.sin(3 * x) + y * z
    coef = torch.zeros(F.fmt_nmono(4), dtype=torch.float64, device="cuda")
    r_out = torch.zeros(n, dtype=torch.float64, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    F.fmt_fit_node_static(4, dev(x), dev(y), dev(z), dev(f), coef, r_out, flags)
    torch.cuda.synchronize()
    c_tree, r_tree, fl_tree = tree_root_fit(x, y, z, f, 4)
    assert int(flags.item()) == fl_tree == F.FMT_FLAG_DEG_CLAMPED
    tol = 1e-10 * np.max(np.abs(f))
    r_s = r_out.cpu().numpy()
    assert np.max(np.abs(r_s - r_tree)) <= tol, np.max(np.abs(r_s - r_tree))
    # the clamped fit in the degree-4 layout: the degree-4 monomials carry zeros,
    # and the cubic itself agrees with the tree path's at the data points
    c_s = coef.cpu().numpy()
    deg4 = [k for k, (l, m, nn) in enumerate((l, m, nn) for l in range(5) for m in range(5 - l)
                                                 for nn in range(5 - l - m)) if l + m + nn == 4]
    assert np.all(c_s[deg4] == 0.0) and np.all(c_tree[deg4] == 0.0)
    pts = np.stack([x, y, z], axis=1)
    key = (0, 0, 0, 0)
    a = TC.node_poly(c_s, 4, key, (0.0, 0.0, 0.0), 1.0, pts)
    b = TC.node_poly(c_tree, 4, key, (0.0, 0.0, 0.0), 1.0, pts)
    assert np.max(np.abs(a - b)) <= tol, np.max(np.abs(a - b))
    with pytest.raises(F.FmtError) as e:
        F.fmt_fit_node_static(F.STATIC_MAX_DEGREE + 1, dev(x), dev(y), dev(z), dev(f), coef, r_out)
    assert e.value.status == F.FMT_EINVAL
    assert "degree" in str(e.value)
