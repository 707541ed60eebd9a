"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test would fail on a plausible mistake in the oracle (a dropped term, a
wrong sign or index, a transposed operand, a wrong frame, a wrong decision):

* rank (number of monomials): printed values in Sec. 3 + brute-force count
* basis order and scaling: Alg. 2 loop order (golden), multinomial identity
* quantisation / octants: exact dyadic values + geometric brute force
* fit: exact rational least squares on tiny inputs (Fractions), and an
  independent SVD-based restatement of Alg. 1/2 on small trees
* invariants: polynomial reproduction (projection, Sec. 2 end), resolution
  of the identity (f = 1), data-point consistency, LS orthogonality on
  leaves, depth-first == breadth-first == OpenMP, permutation invariance
* readings: degree clamp at the root, rank truncation, tau = 0
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_1511_01353_gb300 import workloads as W
from tests import bruteforce as BF

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(t) for t in line.split()])
    return rows


# ---------------------------------------------------------------- rank / basis
def test_nmono_paper_values():
    for p, L in _read_golden("nmono_paper.txt"):
        assert O.nmono(p) == L


def test_nmono_bruteforce_count():
    for p in range(0, 15):
        cnt = sum(1 for t in itertools.product(range(p + 1), repeat=3) if sum(t) <= p)
        assert O.nmono(p) == cnt


def test_monomial_order_golden():
    order = _read_golden("monomial_order_p2.txt")
    # distinct primes make every monomial value unique, so the order is pinned
    u, v, w = 2.0, 3.0, 5.0
    got = O.monomials(2, u, v, w)
    want = [u ** l * v ** m * w ** n / (math.factorial(l) * math.factorial(m) * math.factorial(n))
            for l, m, n in order]
    assert np.array_equal(got, np.array(want))


def test_monomial_multinomial_identity():
    # sum_{l+m+n<=p} u^l v^m w^n/(l!m!n!) = sum_{d<=p} (u+v+w)^d / d!
    rng = np.random.default_rng(3)
    for p in (0, 1, 3, 6, 8, 10):
        for _ in range(5):
            u, v, w = rng.uniform(-1, 1, 3)
            s = u + v + w
            want = sum(s ** d / math.factorial(d) for d in range(p + 1))
            assert abs(O.monomials(p, u, v, w).sum() - want) <= 1e-13 * max(1.0, abs(want))


# ---------------------------------------------------------------- quantisation
def test_quantise_exact_values():
    assert O.quantise(0.0, 1.0, 0.5) == 2 ** 20
    assert O.quantise(0.0, 1.0, 0.5 - 2.0 ** -53) == 2 ** 20 - 1
    assert O.quantise(0.0, 1.0, 0.0) == 0
    assert O.quantise(0.0, 1.0, -0.25) == 0
    assert O.quantise(0.0, 1.0, 1.0) == 2 ** 21 - 1  # upper face clamps into the last cell
    assert O.quantise(0.0, 1.0, 7.0) == 2 ** 21 - 1
    assert O.quantise(-1.0, 2.0, 0.0) == 2 ** 20


def test_octant_bits_match_geometry():
    rng = np.random.default_rng(11)
    pts = rng.uniform(0, 1, (500, 3))
    pts[:50] = np.round(pts[:50] * 64) / 64  # many points exactly on dyadic faces
    for x in pts.reshape(-1):
        q = O.quantise(0.0, 1.0, float(x))
        lo, hi, i = 0.0, 1.0, 0
        for d in range(1, 12):
            c = 0.5 * (lo + hi)
            b = 1 if x >= c else 0
            assert ((q >> (21 - d)) & 1) == b
            lo, hi = (c, hi) if b else (lo, c)


# ---------------------------------------------------------------- single-node fit
def _exact_ls(A_rows, b):
    """Solve the normal equations exactly over the rationals."""
    n, L = len(A_rows), len(A_rows[0])
    G = [[sum(A_rows[i][a] * A_rows[i][c] for i in range(n)) for c in range(L)] for a in range(L)]
    h = [sum(A_rows[i][a] * b[i] for i in range(n)) for a in range(L)]
    M = [G[a] + [h[a]] for a in range(L)]
    for col in range(L):
        piv = next(r for r in range(col, L) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        for r in range(L):
            if r != col and M[r][col] != 0:
                fac = M[r][col] / M[col][col]
                M[r] = [M[r][k] - fac * M[col][k] for k in range(L + 1)]
    return [M[a][L] / M[a][a] for a in range(L)]


@pytest.mark.parametrize("p,n,seed", [(1, 12, 1), (2, 24, 2), (3, 40, 3)])
def test_fit_node_exact_rational(p, n, seed):
    rng = np.random.default_rng(seed)
    u, v, w = (rng.uniform(-1, 1, n) for _ in range(3))
    r = rng.normal(size=n)
    E = BF.exponents(p)
    rows = []
    for i in range(n):
        U, V, Wf = Fraction(float(u[i])), Fraction(float(v[i])), Fraction(float(w[i]))
        rows.append([U ** l * V ** m * Wf ** k / (math.factorial(l) * math.factorial(m) * math.factorial(k))
                     for l, m, k in E])
    b = [Fraction(float(t)) for t in r]
    Fx = np.array([float(t) for t in _exact_ls(rows, b)])
    F, r_new, flags = O.fit_node(p, u, v, w, r)
    assert flags == 0
    A = BF.basis(p, u, v, w)
    cond = np.linalg.cond(A)
    assert np.max(np.abs(F - Fx)) <= 50 * cond * 2.2e-16 * np.max(np.abs(Fx))
    resid_exact = r - A @ Fx
    assert np.max(np.abs(r_new - resid_exact)) <= 50 * cond * 2.2e-16 * np.max(np.abs(r))


def test_fit_node_sign_of_zero_alpha():
    # first column entry alpha = 0 exercises sign(0) = + ; result still exact LS
    u = np.array([0.0, 0.5, -0.5, 0.25, 0.75, -0.25])
    v = np.array([0.1, 0.2, 0.3, -0.4, 0.5, -0.6])
    w = np.zeros(6)
    r = np.array([1.0, 2.0, 0.0, -1.0, 3.0, 0.5])
    F, r_new, _ = O.fit_node(1, u, v, w, r)
    A = np.stack([np.ones(6), w, v, u], axis=1)  # (0,0,0),(0,0,1),(0,1,0),(1,0,0)
    # column of w is zero: rank deficient -> truncated; compare on the (1,v,u) columns
    Fr, *_ = np.linalg.lstsq(A[:, [0, 2, 3]], r, rcond=None)
    assert abs(F[1]) == 0.0
    assert np.allclose(F[[0, 2, 3]], Fr, atol=1e-13)


def test_fit_node_no_cancellation_in_the_reflector():
    # Column 1 of the degree-1 basis is w.  The data make the w column, after
    # the first reflector, almost e_1 with tails of size delta: had the first
    # reflector taken beta = +sign(alpha)*||x|| (x the column from the pivot
    # down), alpha - beta would cancel
    # in the second column.  The dgeqr2 sign (beta = -sign(alpha)*||x||,
    # |alpha - beta| >= |alpha|) never cancels, so the fit stays exact to
    # rounding against rational least squares.
    rng = np.random.default_rng(3)
    n, delta = 24, 1e-7
    t = np.concatenate([[1.0], delta * rng.choice([-1.0, 1.0], n - 2)])
    w = np.concatenate([[0.0], t - t.sum() / (math.sqrt(n) - 1.0)])
    u, v = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    r = rng.normal(size=n)
    rows = [[Fraction(float(a)) ** l * Fraction(float(b)) ** m * Fraction(float(c)) ** k for l, m, k in BF.exponents(1)]
            for a, b, c in zip(u, v, w)]
    Fx = np.array([float(q) for q in _exact_ls(rows, [Fraction(float(q)) for q in r])])
    F, _, flags = O.fit_node(1, u, v, w, r)
    assert flags == 0
    cond = np.linalg.cond(BF.basis(1, u, v, w))
    assert np.max(np.abs(F - Fx)) <= 50 * cond * 2.2e-16 * np.max(np.abs(Fx))


# ---------------------------------------------------------------- whole tree
def _small_case(n=1500, seed=5):
    rng = np.random.default_rng(seed)
    x, y, z = (rng.uniform(0, 1, n) for _ in range(3))
    return x, y, z, W.franke_bj(x, y, z)


def test_tree_matches_independent_svd_restatement():
    x, y, z, f = _small_case()
    p, D, mp, tol = 2, 3, 12, 1e-3
    T = O.fit(x, y, z, f, p, D, mp, tol)
    bf_nodes, bf_r, bf_tau = BF.fmt_tree(x, y, z, f, p, D, mp, tol)
    assert T.tau == bf_tau
    keys = {(int(T.depth[i]),) + tuple(int(a) for a in T.ixyz[i]): i for i in range(T.n_nodes)}
    # no decision here lies near tau, so the node sets must be identical
    for i in range(T.n_nodes):
        for o in range(8):
            if T.child_n[i, o] > 0:
                assert abs(T.child_E[i, o] - T.tau) > 1e-6 * T.tau
    assert set(keys) == set(bf_nodes)
    for k, i in keys.items():
        bn = bf_nodes[k]
        assert T.npts[i] == bn["n"]
        scale = max(1.0, np.max(np.abs(bn["coef"])))
        assert np.max(np.abs(T.coef[i] - bn["coef"])) <= 1e-9 * scale
        assert np.allclose(T.child_E[i], bn["childE"], rtol=1e-7, atol=1e-12)
    assert np.max(np.abs(T.resid - bf_r)) <= 1e-11 * T.maxabs


def test_tree_reaches_max_depth_and_matches_restatement():
    # tau = 0: every child with at least max(L, min_pts) points refines, so the
    # tree is the full octree down to D_max = 2 and no deeper (Alg. 1 stops at
    # the depth limit); the brute-force restatement makes the same decisions
    rng = np.random.default_rng(17)
    n = 4000
    x, y, z = (rng.uniform(0, 1, n) for _ in range(3))
    f = W.franke_bj(x, y, z)
    p, D, mp = 1, 2, 4
    T = O.fit(x, y, z, f, p, D, mp, 0.0)
    counts = np.bincount(T.depth, minlength=D + 1)
    assert counts.tolist() == [1, 8, 64]
    bf_nodes, bf_r, _ = BF.fmt_tree(x, y, z, f, p, D, mp, 0.0)
    keys = {(int(T.depth[i]),) + tuple(int(a) for a in T.ixyz[i]): i for i in range(T.n_nodes)}
    assert set(keys) == set(bf_nodes)
    for k, i in keys.items():
        assert np.max(np.abs(T.coef[i] - bf_nodes[k]["coef"])) <= 1e-10 * max(1.0, np.max(np.abs(T.coef[i])))
    assert np.max(np.abs(T.resid - bf_r)) <= 1e-12 * T.maxabs


def test_sign_symmetry():
    # tau = tol_rel * max|f| is even in f and every other step is odd in the
    # residual, and round-to-nearest is symmetric under negation: fitting -f
    # gives the same tree with every coefficient and residual negated, bitwise
    x, y, z, f = _small_case(2500, 19)
    a = O.fit(x, y, z, f, 3, 3, 20, 1e-4)
    b = O.fit(x, y, z, -f, 3, 3, 20, 1e-4)
    assert a.tau == b.tau == 1e-4 * float(np.max(np.abs(f)))
    assert a.n_nodes == b.n_nodes > 9
    assert np.array_equal(a.depth, b.depth) and np.array_equal(a.ixyz, b.ixyz)
    assert np.array_equal(a.coef, -b.coef)
    assert np.array_equal(a.resid, -b.resid)
    assert np.array_equal(a.child_E, b.child_E)


def test_power_of_two_value_scaling():
    # every step is linear in the residual, E_RMS and tau scale with |f|, and
    # scaling by a power of two commutes with IEEE rounding: fitting 4 f
    # gives the same tree with 4x every coefficient, residual, E and tau
    x, y, z, f = _small_case(2500, 23)
    a = O.fit(x, y, z, f, 3, 3, 20, 1e-4)
    b = O.fit(x, y, z, 4.0 * f, 3, 3, 20, 1e-4)
    assert b.tau == 4.0 * a.tau and a.n_nodes == b.n_nodes > 9
    assert np.array_equal(a.ixyz, b.ixyz) and np.array_equal(a.npts, b.npts)
    assert np.array_equal(4.0 * a.coef, b.coef)
    assert np.array_equal(4.0 * a.resid, b.resid)
    assert np.array_equal(4.0 * a.child_E, b.child_E)


def test_dyadic_rescaling_of_the_domain():
    # doubling the points, lo and side doubles every box centre and halves
    # every frame scale exactly, so the node coordinates (x - c) * s and the
    # quantised codes are bitwise unchanged (Sec. 4 maps each box onto
    # [-1,1]^3): the same tree, coefficients and residual; evaluation at the
    # doubled targets gives the same values
    x, y, z, f = _small_case(2500, 29)
    lo = (0.25, -0.5, 0.125)
    x, y, z = x + lo[0], y + lo[1], z + lo[2]
    a = O.fit(x, y, z, f, 3, 3, 20, 1e-4, lo=lo)
    b = O.fit(2 * x, 2 * y, 2 * z, f, 3, 3, 20, 1e-4, lo=tuple(2 * t for t in lo), side=2.0)
    assert a.n_nodes == b.n_nodes > 9
    assert np.array_equal(a.ixyz, b.ixyz) and np.array_equal(a.npts, b.npts)
    assert np.array_equal(a.coef, b.coef) and np.array_equal(a.resid, b.resid)
    rng = np.random.default_rng(31)
    q = rng.uniform(0, 1, (3, 400)) + np.array(lo)[:, None]
    va, _ = a.evaluate(*q)
    vb, _ = b.evaluate(*(2 * q))
    assert np.array_equal(va, vb)


def test_polynomial_reproduction():
    rng = np.random.default_rng(21)
    p = 3
    n = 3000
    x, y, z = (rng.uniform(0, 1, n) for _ in range(3))
    E = BF.exponents(p)
    cf = rng.normal(size=len(E))

    def g(a, b, c):
        return sum(cf[k] * a ** l * b ** m * c ** q for k, (l, m, q) in enumerate(E))

    f = g(x, y, z)
    T = O.fit(x, y, z, f, p, 4, 10, 1e-6)
    assert T.n_nodes == 1  # residual is roundoff, so nothing refines
    assert np.max(np.abs(T.resid)) <= 1e-12 * T.maxabs
    xq, yq, zq = (rng.uniform(0, 1, 2000) for _ in range(3))
    out, nout = T.evaluate(xq, yq, zq)
    assert nout == 0
    assert np.max(np.abs(out - g(xq, yq, zq))) <= 1e-12 * T.maxabs


def test_resolution_of_identity():
    rng = np.random.default_rng(8)
    n = 800
    x, y, z = (rng.uniform(0, 1, n) for _ in range(3))
    T = O.fit(x, y, z, np.ones(n), 4, 3, 35, 1e-8)
    assert T.n_nodes == 1
    assert abs(T.coef[0, 0] - 1.0) <= 1e-13
    # roundoff scaled by cond(Lambda) ~ 1e3 and by the 1/(l!m!n!) column scaling
    assert np.max(np.abs(T.coef[0, 1:])) <= 1e-11
    xq, yq, zq = (rng.uniform(0, 1, 500) for _ in range(3))
    out, _ = T.evaluate(xq, yq, zq)
    assert np.max(np.abs(out - 1.0)) <= 1e-13


def test_data_point_consistency_and_leaf_orthogonality():
    x, y, z, f = _small_case(2500, 9)
    T = O.fit(x, y, z, f, 3, 3, 20, 1e-4)
    assert T.n_nodes > 9
    out, _ = T.evaluate(x, y, z)
    assert np.max(np.abs(out - (f - T.resid))) <= 1e-12 * T.maxabs
    # on every leaf, the final residual is orthogonal to the leaf's basis
    for i in range(T.n_nodes):
        if np.any(T.child[i] >= 0):
            continue
        d = int(T.depth[i])
        h = 1.0 / 2 ** (d + 1)
        lo = [T.ixyz[i, a] * 2 * h for a in range(3)]
        sel = np.ones(x.shape[0], bool)
        for a, arr in enumerate((x, y, z)):
            sel &= (arr >= lo[a]) & (arr < lo[a] + 2 * h)
        assert sel.sum() == T.npts[i]
        c = [lo[a] + h for a in range(3)]
        A = BF.basis(3, (x[sel] - c[0]) / h, (y[sel] - c[1]) / h, (z[sel] - c[2]) / h)
        g = A.T @ T.resid[sel]
        assert np.linalg.norm(g) <= 1e-11 * np.linalg.norm(A) * max(np.linalg.norm(f[sel]), 1e-300)


def test_dfs_bfs_omp_identical():
    w = W.small()
    a = O.fit(w.x, w.y, w.z, w.f, w.degree, w.max_depth, w.min_pts, w.tol_rel, mode="dfs")
    b = O.fit(w.x, w.y, w.z, w.f, w.degree, w.max_depth, w.min_pts, w.tol_rel, mode="bfs")
    c = O.fit(w.x, w.y, w.z, w.f, w.degree, w.max_depth, w.min_pts, w.tol_rel, mode="omp")
    assert np.array_equal(a.coef, c.coef) and np.array_equal(a.resid, c.resid)
    ka = {(int(a.depth[i]),) + tuple(int(t) for t in a.ixyz[i]): i for i in range(a.n_nodes)}
    kb = {(int(b.depth[i]),) + tuple(int(t) for t in b.ixyz[i]): i for i in range(b.n_nodes)}
    assert set(ka) == set(kb)
    for k in ka:
        assert np.array_equal(a.coef[ka[k]], b.coef[kb[k]])
    assert np.array_equal(a.resid, b.resid)


def test_permutation_invariance():
    x, y, z, f = _small_case(2000, 13)
    a = O.fit(x, y, z, f, 3, 3, 20, 1e-4)
    perm = np.random.default_rng(0).permutation(x.shape[0])
    b = O.fit(x[perm], y[perm], z[perm], f[perm], 3, 3, 20, 1e-4)
    ka = {(int(a.depth[i]),) + tuple(int(t) for t in a.ixyz[i]): i for i in range(a.n_nodes)}
    kb = {(int(b.depth[i]),) + tuple(int(t) for t in b.ixyz[i]): i for i in range(b.n_nodes)}
    assert set(ka) == set(kb)
    for k in ka:
        assert a.npts[ka[k]] == b.npts[kb[k]]
        assert np.max(np.abs(a.coef[ka[k]] - b.coef[kb[k]])) <= 1e-9 * max(1, np.max(np.abs(a.coef[ka[k]])))
    assert np.max(np.abs(a.resid[perm] - b.resid)) <= 1e-12 * a.maxabs


# ---------------------------------------------------------------- readings
def test_root_degree_clamp():
    rng = np.random.default_rng(4)
    x, y, z = (rng.uniform(0, 1, 20) for _ in range(3))
    f = rng.normal(size=20)
    T = O.fit(x, y, z, f, 4, 3, 1, 0.0)
    assert T.n_nodes == 1
    assert T.deg_used[0] == 3 and (T.flags[0] & O.FLAG_DEG_CLAMPED)
    # 20 points, 20 monomials of degree <= 3: the fit interpolates
    assert np.max(np.abs(T.resid)) <= 1e-8 * np.max(np.abs(f))
    # monomials of degree 4 keep a zero coefficient in the degree-4 layout
    deg = np.array([sum(t) for t in BF.exponents(4)])
    assert np.all(T.coef[0, deg == 4] == 0.0)


def test_single_point():
    T = O.fit(np.array([0.3]), np.array([0.6]), np.array([0.9]), np.array([2.5]), 4, 3, 1, 1e-6)
    assert T.n_nodes == 1 and T.deg_used[0] == 0
    assert T.coef[0, 0] == 2.5 and T.resid[0] == 0.0


def test_rank_truncation_on_coplanar_points():
    rng = np.random.default_rng(6)
    n = 400
    x, y = rng.uniform(0, 1, n), rng.uniform(0, 1, n)
    z = np.full(n, 0.25)
    f = 1 + x - 2 * y + 0.5 * x * y
    T = O.fit(x, y, z, f, 2, 2, 10, 1e-6)
    assert T.flags[0] & O.FLAG_RANK
    xq, yq = rng.uniform(0, 1, 100), rng.uniform(0, 1, 100)
    out, _ = T.evaluate(xq, yq, np.full(100, 0.25))
    assert np.max(np.abs(out - (1 + xq - 2 * yq + 0.5 * xq * yq))) <= 1e-10


def test_zero_function_tau_zero():
    rng = np.random.default_rng(7)
    x, y, z = (rng.uniform(0, 1, 300) for _ in range(3))
    T = O.fit(x, y, z, np.zeros(300), 2, 3, 10, 1e-4)
    assert T.tau == 0.0 and T.n_nodes == 1
    assert np.all(T.coef == 0.0)


def test_outside_targets_are_counted_and_extrapolated():
    rng = np.random.default_rng(12)
    x, y, z = (rng.uniform(0, 1, 500) for _ in range(3))
    f = 2 * x - y + 3 * z
    T = O.fit(x, y, z, f, 1, 2, 4, 1e-6)
    xq = np.array([-0.5, 0.5, 1.0, 1.5])
    yq = np.array([0.5, 0.5, 1.0, 0.5])
    zq = np.array([0.5, 2.0, 1.0, 0.5])
    out, nout = T.evaluate(xq, yq, zq)
    assert nout == 3  # the corner (1,1,1) lies on the closed root cube
    assert np.max(np.abs(out - (2 * xq - yq + 3 * zq))) <= 1e-11


def test_invalid_inputs():
    with pytest.raises(ValueError):
        O.fit(np.array([0.1, np.nan]), np.zeros(2), np.zeros(2), np.zeros(2), 1, 1, 1, 1e-3)
    with pytest.raises(ValueError):
        O.fit(np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0), 1, 1, 1, 1e-3)


def test_franke_forms_agree_where_they_must():
    # the two forms differ only in squaring (9y+1), (9z+1): equal when y = z = 0
    xs = np.linspace(0, 1, 17)
    assert np.allclose(W.franke_bj(xs, 0 * xs, 0 * xs), W.franke_paper(xs, 0 * xs, 0 * xs), rtol=0, atol=1e-15)
    # at (2/9, 2/9, 2/9) the first Gaussian of the paper's form is exactly 3/4
    t = 2.0 / 9.0
    rest = 0.75 * math.exp(-(9 * t + 1) ** 2 / 49 - 2 * (9 * t + 1) ** 2 / 10) \
        + 0.5 * math.exp(-0.25 * ((9 * t - 7) ** 2 + (9 * t - 3) ** 2 + (9 * t - 5) ** 2)) \
        - 0.2 * math.exp(-(9 * t - 4) ** 2 - (9 * t - 7) ** 2 - (9 * t - 5) ** 2)
    assert abs(float(W.franke_paper(t, t, t)) - (0.75 + rest)) <= 1e-15


def test_philox_known_answers():
    kat = [((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
           ((0xFFFFFFFF,) * 4, (0xFFFFFFFF, 0xFFFFFFFF), (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
           ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
            (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1))]
    for ctr, key, want in kat:
        got = W.philox4x32_10(tuple(np.array([c], np.uint64) for c in ctr), key)
        assert tuple(int(g[0]) for g in got) == want
