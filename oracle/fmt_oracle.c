/*
 * fmt_oracle.c -- plain, slow FP64 CPU oracle for the free-mesh transform (FMT).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU legs of bench.py (cpu_baseline, --impl reference) may build, load or
 * call this file (__graft_entry__.build() compiles it).  It shares
 * no code, header, table or helper with the CUDA library; the product path
 * never routes through it.
 *
 * What it computes, in the paper's order (Challacombe, "A N-Body Solver for
 * Free Mesh Interpolation", arXiv 1511.01353):
 *
 *   Alg. 1 (FMT_Mesh_to_Tree): translate and dilate the node's points into
 *   the node frame, fit the residual (Alg. 2), order the points by octant,
 *   and for each octant o = 0..7 recurse when its RMS residual exceeds tau
 *   and it holds at least nmono points.  Depth-first, as printed.
 *
 *   Alg. 2 (FMT_Mesh_to_Moments): build the geometric-moment Vandermonde
 *   matrix Lambda_lmn = u^l v^m w^n / (l! m! n!), l+m+n <= p, with l outer,
 *   m middle, n inner; Householder QR (LAPACK dgeqr2 conventions); F =
 *   R^{-1} Q^T f; f <- f - Lambda F.
 *
 *   Sec. 2 end (f(r) = Lambda(r) . F): evaluation at targets, summed over
 *   every existing node on the target's octree path, each in its own frame.
 *
 * Readings of points the paper leaves open (each one documented in the
 * design notes of the repository):
 *   - nmono = (p+1)(p+2)(p+3)/6, the rank stride at p+1 (Sec. 3 gives 84,
 *     286, 680 for L_max = 6, 10, 14).
 *   - tau = tol_rel * max_i |f_i| (relative threshold); refinement is strict
 *     E_RMS > tau, with the point test n_o >= max(nmono, min_pts) and the
 *     child depth <= max_depth.  Decisions with |E - tau| <= 1e-9 tau are
 *     flagged (ORA_FLAG_NEAR_TAU on the created child, near_mask on the parent).
 *   - Octants come from an exact integer quantisation q = floor((x-lo)*S),
 *     S = 2^21/side, clamped to [0, 2^21-1]; child octant at depth d+1 is
 *     bx | by<<1 | bz<<2 with b = bit (20-d) of q.  Within an octant the
 *     parent's order is kept (stable).
 *   - Node frame: h = side * 2^-(d+1), centre c = lo + (2i+1)*h, scale
 *     s = 1/h, u = (x - c) * s, computed from global coordinates with no
 *     fused multiply-add (this file is compiled with -ffp-contract=off).
 *   - Root with N < nmono: the root degree is clamped to the largest p' with
 *     nmono(p') <= N (ORA_FLAG_DEG_CLAMPED); coefficients stay in the
 *     degree-p layout with zeros for the dropped monomials.
 *   - Rank deficiency: a column with |R_jj| <= 64*nmono*eps*max|R_kk|
 *     (eps = 2^-52) gets F_j = 0 and ORA_FLAG_RANK; it is deleted from
 *     [R | Q^T f] and the rest is re-triangularised before back substitution,
 *     so the kept coefficients are the least-squares fit over kept columns.
 *   - Householder: beta = -sign(alpha) * sqrt(alpha^2 + |x|^2) with sign(0)=+;
 *     a column with |x| = 0 gets tau = 0 (no reflection).
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_QBITS 21
#define ORA_QMAX ((1u << ORA_QBITS) - 1u)

#define ORA_FLAG_NEAR_TAU 1
#define ORA_FLAG_RANK 2
#define ORA_FLAG_DEG_CLAMPED 4

#define ORA_OK 0
#define ORA_EINVAL 1
#define ORA_ENOMEM 2

typedef struct {
  int32_t depth, deg_used, flags;
  uint32_t ix, iy, iz;
  int64_t n;
  int64_t parent;
  int64_t child[8];
  double child_E[8];
  int64_t child_n[8];
  uint32_t near_mask, refine_mask;
  double *coef; /* nmono(p) doubles, Alg. 2 order */
} ora_node;

typedef struct {
  ora_node *v;
  int64_t len, cap;
} ora_nodelist;

typedef struct ora_tree {
  int degree, nmono, max_depth, min_pts;
  double tol_rel, tau, maxabs, lo[3], side;
  int64_t npts;
  double *resid; /* final residual, input order */
  ora_nodelist nodes;
} ora_tree;

/* ---- Sec. 2: rank stride l3_i = i(i+1)(i+2)/6; nmono = l3_{p+1} ---- */
int ora_nmono(int p) {
  if (p < 0) return 0;
  return (p + 1) * (p + 2) * (p + 3) / 6;
}

static double ora_factorial(int k) {
  double f = 1.0;
  for (int i = 2; i <= k; ++i) f *= (double)i;
  return f;
}

static double ora_ipow(double a, int k) {
  double r = 1.0;
  for (int i = 0; i < k; ++i) r *= a;
  return r;
}

/* ---- Sec. 2 / Alg. 2: geometric moments in the l, m, n loop order ---- */
void ora_monomials(int p, double u, double v, double w, double *out) {
  int k = 0;
  for (int l = 0; l <= p; ++l)
    for (int m = 0; m <= p - l; ++m)
      for (int n = 0; n <= p - l - m; ++n)
        out[k++] = ora_ipow(u, l) * ora_ipow(v, m) * ora_ipow(w, n) /
                   (ora_factorial(l) * ora_factorial(m) * ora_factorial(n));
}

/* Position of monomial (l,m,n) of total degree <= q inside the degree-p list. */
static void ora_index_map(int p, int q, int *map) {
  int k = 0, kq = 0;
  for (int l = 0; l <= p; ++l)
    for (int m = 0; m <= p - l; ++m)
      for (int n = 0; n <= p - l - m; ++n) {
        if (l + m + n <= q) map[kq++] = k;
        ++k;
      }
}

/* ---- exact integer quantisation of one coordinate ---- */
uint32_t ora_quantise(double lo, double side, double x) {
  double S = 2097152.0 / side; /* 2^21 / side */
  double t = (x - lo) * S;
  if (!(t >= 0.0)) return 0u;
  if (t >= 2097152.0) return ORA_QMAX;
  return (uint32_t)floor(t);
}

/* node frame (Alg. 1 first step; Sec. 4 maps each octant onto [-1,1]^3) */
static void ora_frame(const ora_tree *T, int depth, uint32_t i, int axis, double *c, double *s) {
  double h = ldexp(T->side, -(depth + 1));
  *c = T->lo[axis] + (double)(2u * i + 1u) * h;
  *s = 1.0 / h;
}

/* ---- Householder QR (dgeqr2 conventions), column-major A[n x L] ---- */
static void ora_householder_qr(int64_t n, int L, double *A, double *tau) {
  for (int j = 0; j < L; ++j) {
    double *aj = A + (int64_t)j * n;
    double alpha = aj[j];
    double xn2 = 0.0;
    for (int64_t i = j + 1; i < n; ++i) xn2 += aj[i] * aj[i];
    if (xn2 == 0.0) {
      tau[j] = 0.0;
      continue;
    }
    double h = sqrt(alpha * alpha + xn2);
    double beta = (alpha >= 0.0) ? -h : h;
    tau[j] = (beta - alpha) / beta;
    double scal = 1.0 / (alpha - beta);
    for (int64_t i = j + 1; i < n; ++i) aj[i] *= scal;
    aj[j] = beta;
    for (int k = j + 1; k < L; ++k) {
      double *ak = A + (int64_t)k * n;
      double w = ak[j];
      for (int64_t i = j + 1; i < n; ++i) w += aj[i] * ak[i];
      w *= tau[j];
      ak[j] -= w;
      for (int64_t i = j + 1; i < n; ++i) ak[i] -= w * aj[i];
    }
  }
}

/* y <- Q^T y, applying H_0, H_1, ... in order (v_j(j) = 1 implicit) */
static void ora_apply_qt(int64_t n, int L, const double *A, const double *tau, double *y) {
  for (int j = 0; j < L; ++j) {
    if (tau[j] == 0.0) continue;
    const double *aj = A + (int64_t)j * n;
    double w = y[j];
    for (int64_t i = j + 1; i < n; ++i) w += aj[i] * y[i];
    w *= tau[j];
    y[j] -= w;
    for (int64_t i = j + 1; i < n; ++i) y[i] -= w * aj[i];
  }
}

/* Plain back substitution on an upper triangle with leading dimension ld. */
static void ora_back_subst(int L, const double *A, int64_t ld, const double *y, double *F, double thresh) {
  for (int j = L - 1; j >= 0; --j) {
    double rjj = A[(int64_t)j * ld + j];
    if (fabs(rjj) <= thresh) {
      F[j] = 0.0;
      continue;
    }
    double s = y[j];
    for (int k = j + 1; k < L; ++k) s -= A[(int64_t)k * ld + j] * F[k];
    F[j] = s / rjj;
  }
}

/*
 * F = R^{-1} y with the rank rule.  Columns j with |R_jj| <= 64*L*eps*max|R_kk|
 * depend (numerically) on the columns before them; they get F_j = 0 and are
 * deleted from [R | y], the remaining L x (Lk+1) matrix is re-triangularised
 * by Householder QR, and the kept coefficients come from that triangle, which
 * is the least-squares solution over the kept columns.  Returns 1 if any
 * column was dropped.
 */
static int ora_back_solve(int64_t n, int L, const double *A, const double *y, double *F) {
  double rmax = 0.0;
  for (int j = 0; j < L; ++j) {
    double a = fabs(A[(int64_t)j * n + j]);
    if (a > rmax) rmax = a;
  }
  double thresh = 64.0 * (double)L * DBL_EPSILON * rmax;
  int ndrop = 0;
  for (int j = 0; j < L; ++j)
    if (fabs(A[(int64_t)j * n + j]) <= thresh) ++ndrop;
  if (ndrop == 0) {
    ora_back_subst(L, A, n, y, F, -1.0);
    return 0;
  }
  int Lk = L - ndrop;
  double *M = (double *)calloc((size_t)L * (size_t)(Lk + 1), sizeof(double));
  double *tau = (double *)malloc(sizeof(double) * (size_t)(Lk + 1));
  double *Fk = (double *)malloc(sizeof(double) * (size_t)(Lk > 0 ? Lk : 1));
  int *keep = (int *)malloc(sizeof(int) * (size_t)(Lk > 0 ? Lk : 1));
  if (!M || !tau || !Fk || !keep) { /* out of memory: fall back to zeros */
    for (int j = 0; j < L; ++j) F[j] = 0.0;
    free(M); free(tau); free(Fk); free(keep);
    return 1;
  }
  int c = 0;
  for (int j = 0; j < L; ++j) {
    if (fabs(A[(int64_t)j * n + j]) <= thresh) continue;
    keep[c] = j;
    for (int i = 0; i <= j; ++i) M[(int64_t)c * L + i] = A[(int64_t)j * n + i];
    ++c;
  }
  for (int i = 0; i < L; ++i) M[(int64_t)Lk * L + i] = y[i];
  ora_householder_qr(L, Lk + 1 <= L ? Lk + 1 : L, M, tau);
  ora_back_subst(Lk, M, L, M + (int64_t)Lk * L, Fk, thresh);
  for (int j = 0; j < L; ++j) F[j] = 0.0;
  for (int i = 0; i < Lk; ++i) F[keep[i]] = Fk[i];
  free(M); free(tau); free(Fk); free(keep);
  return 1;
}

/*
 * Alg. 2 on one point set in node coordinates (u,v,w): fit r by least
 * squares over the degree-q basis, subtract, return F (length nmono(q)).
 * Returns ORA_FLAG_RANK when the back substitution truncated, -1 on ENOMEM.
 */
int ora_fit_node(int q, int64_t n, const double *u, const double *v, const double *w,
                 double *r, double *F) {
  int L = ora_nmono(q);
  if (n < 1 || L < 1) return -1;
  double *A = (double *)malloc(sizeof(double) * (size_t)n * (size_t)L);
  double *tau = (double *)malloc(sizeof(double) * (size_t)L);
  double *y = (double *)malloc(sizeof(double) * (size_t)n);
  double *row = (double *)malloc(sizeof(double) * (size_t)L);
  if (!A || !tau || !y || !row) {
    free(A); free(tau); free(y); free(row);
    return -1;
  }
  for (int64_t i = 0; i < n; ++i) {
    ora_monomials(q, u[i], v[i], w[i], row);
    for (int k = 0; k < L; ++k) A[(int64_t)k * n + i] = row[k];
  }
  int Lq = (n < L) ? (int)n : L; /* never happens after the degree clamp */
  ora_householder_qr(n, Lq, A, tau);
  memcpy(y, r, sizeof(double) * (size_t)n);
  ora_apply_qt(n, Lq, A, tau, y);
  for (int k = 0; k < L; ++k) F[k] = 0.0;
  int flags = ora_back_solve(n, Lq, A, y, F) ? ORA_FLAG_RANK : 0;
  /* f <- f - Lambda F with the same basis values */
  for (int64_t i = 0; i < n; ++i) {
    ora_monomials(q, u[i], v[i], w[i], row);
    double s = 0.0;
    for (int k = 0; k < L; ++k) s += row[k] * F[k];
    r[i] -= s;
  }
  free(A); free(tau); free(y); free(row);
  return flags;
}

/* ---------------- tree ---------------- */
typedef struct {
  const ora_tree *T;
  const double *x, *y, *z;
  const uint32_t *qx, *qy, *qz;
  double *r; /* residual, input order, updated in place */
  int parallel;
} ora_ctx;

static int ora_push(ora_nodelist *L, const ora_node *nd) {
  if (L->len == L->cap) {
    int64_t nc = L->cap ? 2 * L->cap : 16;
    ora_node *nv = (ora_node *)realloc(L->v, sizeof(ora_node) * (size_t)nc);
    if (!nv) return -1;
    L->v = nv;
    L->cap = nc;
  }
  L->v[L->len++] = *nd;
  return 0;
}

static void ora_free_list(ora_nodelist *L) {
  for (int64_t i = 0; i < L->len; ++i) free(L->v[i].coef);
  free(L->v);
  L->v = NULL;
  L->len = L->cap = 0;
}

/* Fit one node (Alg. 1 first two steps) and fill its child statistics. */
static int ora_fit_one(const ora_ctx *C, ora_node *nd, const int64_t *idx, int64_t n,
                       int64_t *child_count, int64_t **child_idx) {
  const ora_tree *T = C->T;
  int p = T->degree;
  int q = p;
  nd->flags &= ORA_FLAG_NEAR_TAU;
  if (nd->depth == 0 && n < T->nmono) {
    q = -1;
    while (ora_nmono(q + 1) <= n) ++q;
    nd->flags |= ORA_FLAG_DEG_CLAMPED;
  }
  nd->deg_used = q;
  nd->n = n;
  nd->coef = (double *)calloc((size_t)T->nmono, sizeof(double));
  double *u = (double *)malloc(sizeof(double) * (size_t)n);
  double *v = (double *)malloc(sizeof(double) * (size_t)n);
  double *w = (double *)malloc(sizeof(double) * (size_t)n);
  double *r = (double *)malloc(sizeof(double) * (size_t)n);
  int Lq = ora_nmono(q);
  double *F = (double *)malloc(sizeof(double) * (size_t)(Lq > 0 ? Lq : 1));
  int *map = (int *)malloc(sizeof(int) * (size_t)(Lq > 0 ? Lq : 1));
  if (!nd->coef || !u || !v || !w || !r || !F || !map) {
    free(u); free(v); free(w); free(r); free(F); free(map);
    return -1;
  }
  double cx, sx, cy, sy, cz, sz;
  ora_frame(T, nd->depth, nd->ix, 0, &cx, &sx);
  ora_frame(T, nd->depth, nd->iy, 1, &cy, &sy);
  ora_frame(T, nd->depth, nd->iz, 2, &cz, &sz);
  for (int64_t i = 0; i < n; ++i) {
    int64_t g = idx[i];
    u[i] = (C->x[g] - cx) * sx;
    v[i] = (C->y[g] - cy) * sy;
    w[i] = (C->z[g] - cz) * sz;
    r[i] = C->r[g];
  }
  if (q >= 0) {
    int fl = ora_fit_node(q, n, u, v, w, r, F);
    if (fl < 0) {
      free(u); free(v); free(w); free(r); free(F); free(map);
      return -1;
    }
    nd->flags |= fl;
    ora_index_map(p, q, map);
    for (int k = 0; k < Lq; ++k) nd->coef[map[k]] = F[k];
  }
  for (int64_t i = 0; i < n; ++i) C->r[idx[i]] = r[i];

  /* FMT_Ordered_by_Octant: stable partition by the child octant bits */
  int shift = ORA_QBITS - 1 - nd->depth;
  for (int o = 0; o < 8; ++o) child_count[o] = 0;
  if (shift >= 0) {
    for (int64_t i = 0; i < n; ++i) {
      int64_t g = idx[i];
      int o = (int)(((C->qx[g] >> shift) & 1u) | (((C->qy[g] >> shift) & 1u) << 1) |
                    (((C->qz[g] >> shift) & 1u) << 2));
      child_count[o]++;
    }
  }
  for (int o = 0; o < 8; ++o) {
    child_idx[o] = (int64_t *)malloc(sizeof(int64_t) * (size_t)(child_count[o] > 0 ? child_count[o] : 1));
    if (!child_idx[o]) return -1;
  }
  int64_t fill[8] = {0};
  double S[8] = {0};
  if (shift >= 0) {
    for (int64_t i = 0; i < n; ++i) {
      int64_t g = idx[i];
      int o = (int)(((C->qx[g] >> shift) & 1u) | (((C->qy[g] >> shift) & 1u) << 1) |
                    (((C->qz[g] >> shift) & 1u) << 2));
      child_idx[o][fill[o]++] = g;
    }
  }
  /* Alg. 1 loop body: E_RMS over each octant's points, in their order */
  for (int o = 0; o < 8; ++o) {
    for (int64_t i = 0; i < child_count[o]; ++i) {
      double e = C->r[child_idx[o][i]];
      S[o] += e * e;
    }
    nd->child_n[o] = child_count[o];
    nd->child_E[o] = child_count[o] > 0 ? sqrt(S[o] / (double)child_count[o]) : 0.0;
    nd->child[o] = -1;
  }
  nd->near_mask = nd->refine_mask = 0;
  int64_t nmin = T->min_pts > T->nmono ? T->min_pts : T->nmono;
  for (int o = 0; o < 8; ++o) {
    if (child_count[o] == 0) continue;
    double E = nd->child_E[o];
    int deep_ok = (nd->depth + 1 <= T->max_depth) && (shift >= 0);
    int pts_ok = child_count[o] >= nmin;
    if (deep_ok && pts_ok && fabs(E - T->tau) <= 1e-9 * T->tau) nd->near_mask |= 1u << o;
    if (deep_ok && pts_ok && E > T->tau) nd->refine_mask |= 1u << o;
  }
  free(u); free(v); free(w); free(r); free(F); free(map);
  return 0;
}

/* Alg. 1, depth first.  Appends the subtree (preorder) to out. */
static int ora_recurse(const ora_ctx *C, ora_node nd, const int64_t *idx, int64_t n, ora_nodelist *out) {
  int64_t cc[8];
  int64_t *ci[8] = {0};
  int rc = ora_fit_one(C, &nd, idx, n, cc, ci);
  if (rc) {
    for (int o = 0; o < 8; ++o) free(ci[o]);
    free(nd.coef);
    return rc;
  }
  int64_t self = out->len;
  if (ora_push(out, &nd)) {
    for (int o = 0; o < 8; ++o) free(ci[o]);
    free(nd.coef);
    return -1;
  }
  ora_nodelist sub[8];
  int subrc[8];
  memset(sub, 0, sizeof(sub));
  for (int o = 0; o < 8; ++o) subrc[o] = 0;
  for (int o = 0; o < 8; ++o) {
    if (!(nd.refine_mask & (1u << o))) continue;
    ora_node ch;
    memset(&ch, 0, sizeof(ch));
    ch.depth = nd.depth + 1;
    ch.ix = 2u * nd.ix + (uint32_t)(o & 1);
    ch.iy = 2u * nd.iy + (uint32_t)((o >> 1) & 1);
    ch.iz = 2u * nd.iz + (uint32_t)((o >> 2) & 1);
    ch.flags = (nd.near_mask & (1u << o)) ? ORA_FLAG_NEAR_TAU : 0;
    ch.parent = -1;
#ifdef _OPENMP
#pragma omp task shared(sub, subrc, ci, cc) firstprivate(ch, o) if (C->parallel && cc[o] > 2048)
#endif
    subrc[o] = ora_recurse(C, ch, ci[o], cc[o], &sub[o]);
  }
#ifdef _OPENMP
#pragma omp taskwait
#endif
  int err = 0;
  for (int o = 0; o < 8; ++o) {
    free(ci[o]);
    if (subrc[o]) err = subrc[o];
    if (!(nd.refine_mask & (1u << o))) continue;
    int64_t base = out->len;
    for (int64_t i = 0; i < sub[o].len; ++i) {
      ora_node c = sub[o].v[i];
      c.parent = (c.parent < 0) ? self : c.parent + base;
      for (int k = 0; k < 8; ++k)
        if (c.child[k] >= 0) c.child[k] += base;
      if (ora_push(out, &c)) err = -1;
    }
    if (sub[o].len > 0) out->v[self].child[o] = base;
    free(sub[o].v); /* coefficient buffers now owned by out */
  }
  return err;
}

static int ora_prepare(ora_tree *T, ora_ctx *C, int64_t n, const double *x, const double *y,
                       const double *z, const double *f, uint32_t **qx, uint32_t **qy, uint32_t **qz) {
  double M = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    if (!isfinite(x[i]) || !isfinite(y[i]) || !isfinite(z[i]) || !isfinite(f[i])) return ORA_EINVAL;
    double a = fabs(f[i]);
    if (a > M) M = a;
  }
  T->maxabs = M;
  T->tau = T->tol_rel * M;
  T->npts = n;
  T->resid = (double *)malloc(sizeof(double) * (size_t)n);
  *qx = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  *qy = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  *qz = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
  if (!T->resid || !*qx || !*qy || !*qz) return ORA_ENOMEM;
  for (int64_t i = 0; i < n; ++i) {
    T->resid[i] = f[i]; /* r := f */
    (*qx)[i] = ora_quantise(T->lo[0], T->side, x[i]);
    (*qy)[i] = ora_quantise(T->lo[1], T->side, y[i]);
    (*qz)[i] = ora_quantise(T->lo[2], T->side, z[i]);
  }
  C->T = T;
  C->x = x; C->y = y; C->z = z;
  C->qx = *qx; C->qy = *qy; C->qz = *qz;
  C->r = T->resid;
  return ORA_OK;
}

/* Level-synchronous (breadth-first) driver over the same node routine; used
 * only to pin that siblings are independent once the parent is fitted. */
static int ora_bfs(const ora_ctx *C, int64_t n, ora_nodelist *out) {
  typedef struct { int64_t node; int64_t *idx; int64_t n; } item;
  item *cur = (item *)malloc(sizeof(item));
  int64_t ncur = 1;
  if (!cur) return -1;
  cur[0].idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  if (!cur[0].idx) return -1;
  for (int64_t i = 0; i < n; ++i) cur[0].idx[i] = i;
  cur[0].n = n;
  ora_node root;
  memset(&root, 0, sizeof(root));
  root.parent = -1;
  if (ora_push(out, &root)) return -1;
  cur[0].node = 0;
  while (ncur > 0) {
    item *nxt = (item *)malloc(sizeof(item) * (size_t)(8 * ncur));
    int64_t nn = 0;
    for (int64_t a = 0; a < ncur; ++a) {
      int64_t cc[8];
      int64_t *ci[8] = {0};
      ora_node nd = out->v[cur[a].node];
      if (ora_fit_one(C, &nd, cur[a].idx, cur[a].n, cc, ci)) return -1;
      out->v[cur[a].node] = nd;
      free(cur[a].idx);
      for (int o = 0; o < 8; ++o) {
        if (!(nd.refine_mask & (1u << o))) {
          free(ci[o]);
          continue;
        }
        ora_node ch;
        memset(&ch, 0, sizeof(ch));
        ch.depth = nd.depth + 1;
        ch.ix = 2u * nd.ix + (uint32_t)(o & 1);
        ch.iy = 2u * nd.iy + (uint32_t)((o >> 1) & 1);
        ch.iz = 2u * nd.iz + (uint32_t)((o >> 2) & 1);
        ch.flags = (nd.near_mask & (1u << o)) ? ORA_FLAG_NEAR_TAU : 0;
        ch.parent = cur[a].node;
        for (int k = 0; k < 8; ++k) ch.child[k] = -1;
        if (ora_push(out, &ch)) return -1;
        out->v[cur[a].node].child[o] = out->len - 1;
        nxt[nn].node = out->len - 1;
        nxt[nn].idx = ci[o];
        nxt[nn].n = cc[o];
        ++nn;
      }
    }
    free(cur);
    cur = nxt;
    ncur = nn;
  }
  free(cur);
  return 0;
}

/*
 * Fit the whole tree.  mode 0: depth-first serial (Alg. 1 as printed);
 * mode 1: depth-first with OpenMP tasks over sibling subtrees (identical
 * results, each node stays serial); mode 2: breadth-first.
 */
int ora_fit(int degree, int max_depth, int min_pts, double tol_rel, const double *lo, double side,
            int64_t n, const double *x, const double *y, const double *z, const double *f, int mode,
            ora_tree **out) {
  *out = NULL;
  if (degree < 0 || max_depth < 0 || max_depth > ORA_QBITS || n < 1 || !(side > 0.0) ||
      !(tol_rel >= 0.0) || !isfinite(side) || !isfinite(tol_rel))
    return ORA_EINVAL;
  ora_tree *T = (ora_tree *)calloc(1, sizeof(ora_tree));
  if (!T) return ORA_ENOMEM;
  T->degree = degree;
  T->nmono = ora_nmono(degree);
  T->max_depth = max_depth;
  T->min_pts = min_pts;
  T->tol_rel = tol_rel;
  T->lo[0] = lo[0]; T->lo[1] = lo[1]; T->lo[2] = lo[2];
  T->side = side;
  ora_ctx C;
  memset(&C, 0, sizeof(C));
  uint32_t *qx = NULL, *qy = NULL, *qz = NULL;
  int rc = ora_prepare(T, &C, n, x, y, z, f, &qx, &qy, &qz);
  if (rc) {
    free(qx); free(qy); free(qz);
    free(T->resid);
    free(T);
    return rc;
  }
  C.parallel = (mode == 1);
  if (mode == 2) {
    rc = ora_bfs(&C, n, &T->nodes) ? ORA_ENOMEM : ORA_OK;
  } else {
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!idx) rc = ORA_ENOMEM;
    else {
      for (int64_t i = 0; i < n; ++i) idx[i] = i;
      ora_node root;
      memset(&root, 0, sizeof(root));
      root.parent = -1;
      int e = 0;
#ifdef _OPENMP
      if (C.parallel) {
#pragma omp parallel
#pragma omp single
        e = ora_recurse(&C, root, idx, n, &T->nodes);
      } else
#endif
        e = ora_recurse(&C, root, idx, n, &T->nodes);
      rc = e ? ORA_ENOMEM : ORA_OK;
      free(idx);
    }
  }
  free(qx); free(qy); free(qz);
  if (rc) {
    ora_free_list(&T->nodes);
    free(T->resid);
    free(T);
    return rc;
  }
  *out = T;
  return ORA_OK;
}

int64_t ora_num_nodes(const ora_tree *T) { return T->nodes.len; }
double ora_tau(const ora_tree *T) { return T->tau; }
double ora_maxabs(const ora_tree *T) { return T->maxabs; }

void ora_get_nodes(const ora_tree *T, int32_t *depth, uint32_t *ixyz, int64_t *npts, int32_t *flags,
                   int32_t *deg_used, int64_t *parent, int64_t *child, double *child_E, int64_t *child_n,
                   uint32_t *near_mask, uint32_t *refine_mask, double *coef) {
  for (int64_t i = 0; i < T->nodes.len; ++i) {
    const ora_node *nd = &T->nodes.v[i];
    depth[i] = nd->depth;
    ixyz[3 * i + 0] = nd->ix;
    ixyz[3 * i + 1] = nd->iy;
    ixyz[3 * i + 2] = nd->iz;
    npts[i] = nd->n;
    flags[i] = nd->flags;
    deg_used[i] = nd->deg_used;
    parent[i] = nd->parent;
    for (int o = 0; o < 8; ++o) {
      child[8 * i + o] = nd->child[o];
      child_E[8 * i + o] = nd->child_E[o];
      child_n[8 * i + o] = nd->child_n[o];
    }
    near_mask[i] = nd->near_mask;
    refine_mask[i] = nd->refine_mask;
    memcpy(coef + (size_t)i * (size_t)T->nmono, nd->coef, sizeof(double) * (size_t)T->nmono);
  }
}

void ora_get_residual(const ora_tree *T, double *r) {
  memcpy(r, T->resid, sizeof(double) * (size_t)T->npts);
}

/* f(r) = sum over the target's existing octree path of Lambda(u_d) . F_d */
int ora_eval(const ora_tree *T, int64_t m, const double *xq, const double *yq, const double *zq,
             double *out, int64_t *n_outside) {
  int64_t outside = 0;
  double *row = (double *)malloc(sizeof(double) * (size_t)T->nmono);
  if (!row) return ORA_ENOMEM;
  for (int64_t t = 0; t < m; ++t) {
    double x = xq[t], y = yq[t], z = zq[t];
    if (!(x >= T->lo[0] && x <= T->lo[0] + T->side && y >= T->lo[1] && y <= T->lo[1] + T->side &&
          z >= T->lo[2] && z <= T->lo[2] + T->side))
      ++outside;
    uint32_t qx = ora_quantise(T->lo[0], T->side, x);
    uint32_t qy = ora_quantise(T->lo[1], T->side, y);
    uint32_t qz = ora_quantise(T->lo[2], T->side, z);
    double acc = 0.0;
    int64_t node = T->nodes.len > 0 ? 0 : -1;
    while (node >= 0) {
      const ora_node *nd = &T->nodes.v[node];
      double cx, sx, cy, sy, cz, sz;
      ora_frame(T, nd->depth, nd->ix, 0, &cx, &sx);
      ora_frame(T, nd->depth, nd->iy, 1, &cy, &sy);
      ora_frame(T, nd->depth, nd->iz, 2, &cz, &sz);
      ora_monomials(T->degree, (x - cx) * sx, (y - cy) * sy, (z - cz) * sz, row);
      double s = 0.0;
      for (int k = 0; k < T->nmono; ++k) s += row[k] * nd->coef[k];
      acc += s;
      int shift = ORA_QBITS - 1 - nd->depth;
      if (shift < 0) break;
      int o = (int)(((qx >> shift) & 1u) | (((qy >> shift) & 1u) << 1) | (((qz >> shift) & 1u) << 2));
      node = nd->child[o];
    }
    out[t] = acc;
  }
  free(row);
  if (n_outside) *n_outside = outside;
  return ORA_OK;
}

void ora_free(ora_tree *T) {
  if (!T) return;
  ora_free_list(&T->nodes);
  free(T->resid);
  free(T);
}

int ora_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
