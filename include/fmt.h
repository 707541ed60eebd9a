/*
 * fmt.h -- C ABI of the GB300 free-mesh transform (FMT) library, libfmt.so.
 *
 * The free-mesh transform (Challacombe, "A N-Body Solver for Free Mesh
 * Interpolation", arXiv 1511.01353) fits scattered samples f(x_i) with a
 * tree of local polynomials: Alg. 1 recursively splits an octree, Alg. 2 fits
 * each node's current residual by least squares over the geometric moments
 * Lambda_lmn = u^l v^m w^n / (l! m! n!), l+m+n <= p, and hands the residual
 * to the children whose RMS error is still above tau.  The interpolant at a
 * target is the sum of the polynomials of the nodes on its octree path
 * (Sec. 2, end: f(r) = Lambda(r) . F).
 *
 * Conventions shared by every call:
 *  - All functions are extern "C", take plain pointers and sizes, and never
 *    throw.  They return fmt_status; details of the last failure are in
 *    fmt_last_error().
 *  - "device" pointers are CUDA device (or managed) memory on the current
 *    device; "host" pointers are ordinary host memory.
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream.  Work is enqueued on it asynchronously; calls marked
 *    "synchronises" wait for the stream before returning.
 *  - Caller-owned inputs must stay valid and unmodified until the stream has
 *    reached the call.  The tree owns its sorted copies, scratch and
 *    coefficients; fmt_tree_free releases them.
 *  - Errors are sticky per tree: after a device-side error every later call
 *    on that tree returns the same status.
 *  - Threads: calls on different trees may run at the same time from
 *    different host threads, each on its own stream (the library's shared
 *    state -- launch limits, the tuning table, the profile counters, the
 *    memory pool -- is guarded).  One tree is used by one thread at a time.
 *    fmt_fit_node_static is the exception: its calls share one scratch
 *    array per device and must be ordered (see there).
 *    fmt_tune_set and fmt_autotune change the table that later fits read, so
 *    they belong between fits, not beside them.
 *  - Precision: everything on the FP64 path is IEEE binary64.  The
 *    quantisation and node-frame arithmetic use no fused multiply-add so the
 *    tree structure is bit-reproducible.  The mixed path (FMT_MIXED) forms
 *    the least-squares projections with BF16 tensor-core products and wins
 *    the accuracy back in FP64; see fit_level.
 */
#ifndef FMT_H
#define FMT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FMT_OK = 0,
  FMT_EINVAL = 1,    /* bad argument, non-finite input, or call out of order */
  FMT_ENOMEM = 2,    /* device or host allocation failed */
  FMT_ECUDA = 3,     /* a CUDA runtime call failed */
  FMT_ETIMEOUT = 4,  /* a bounded device wait ran out (mixed path) */
  FMT_EINTERNAL = 5  /* a device-side consistency check failed */
} fmt_status;

#define FMT_FP64 0  /* FP64 path: Householder QR of every node in binary64 */
#define FMT_MIXED 1 /* split-BF16 tensor-core Gram + FP64 factorisation and refinement */
#define FMT_MIXED_MAX_DEGREE 9 /* nodes of higher degree skip the tensor-core tier */
#define FMT_MIXED_FP64_MAX_DEGREE 10 /* nodes of higher degree take Householder (see fit_level) */
#define FMT_MIXED_MAX_SWEEPS 3

#define FMT_MAX_DEPTH 21  /* 21 bits per axis in the Morton code */
#define FMT_MAX_DEGREE 14 /* nmono(14) = 680, the largest order in Sec. 3 */

/* Node flags (fmt_tree_export node_flags[]). */
#define FMT_FLAG_NEAR_TAU 1     /* created by a decision with |E - tau| <= 1e-9 tau */
#define FMT_FLAG_RANK 2         /* back substitution dropped dependent columns */
#define FMT_FLAG_DEG_CLAMPED 4  /* root with N < nmono: degree lowered */
#define FMT_FLAG_MIXED 8        /* fitted by the mixed-precision path */
#define FMT_FLAG_MIXED_SLOW 16  /* mixed path: refinement not converged (tensor-core tier, or both tiers) */
#define FMT_FLAG_MIXED_PIVOT 32 /* mixed path: a Cholesky pivot too small (tensor-core tier, or both tiers) */
#define FMT_FLAG_MIXED_FP64 64  /* mixed path: fitted by its FP64 normal-equations tier (with FMT_FLAG_MIXED) */

/*
 * Parameters of Alg. 1 (L, nmono, tau and the root box P) plus the depth and
 * point-count limits of the benchmark configurations.
 *   degree     p, 0 <= p <= 14; nmono = (p+1)(p+2)(p+3)/6 (Sec. 3 prints 84,
 *              286, 680 for p = 6, 10, 14).
 *   max_depth  deepest octree level, 0 <= max_depth <= 21 (root = 0).
 *   min_pts    an octant becomes a child only if it holds at least
 *              max(nmono, min_pts) points (Alg. 1 requires n_o >= nmono).
 *   precision  FMT_FP64 or FMT_MIXED (fit_level describes both).
 *   tol_rel    tau = tol_rel * max_i |f_i| (>= 0); an octant is refined when
 *              its RMS residual E_RMS > tau (strict, Alg. 1).
 *   lo, side   root cube [lo, lo+side)^3, side > 0.  Points and targets
 *              outside it are clamped into the boundary cells.
 *   chunk_rows rows per QR work item for large nodes (multiple of 64);
 *              0 picks a size from the number of active points.
 *   sweeps     FMT_MIXED only: at most this many FP64 refinement sweeps after
 *              the first solve: 1..3 (FMT_MIXED_MAX_SWEEPS), 0 selects 3, -1
 *              none (then no convergence test either); a node that passes
 *              the acceptance tests after an earlier sweep skips the rest.
 *              Ignored for FP64.
 *   options    bit set: FMT_OPT_GRAPH captures the launches of each
 *              fit_level in a CUDA graph (one graph per level step) and
 *              launches that; other bits must be 0.
 */
typedef struct {
  int32_t degree;
  int32_t max_depth;
  int32_t min_pts;
  int32_t precision;
  double tol_rel;
  double lo[3];
  double side;
  int64_t chunk_rows;
  int32_t sweeps;
  int32_t options;
} fmt_params;

/* fmt_params.options bits.  FMT_OPT_GRAPH: fit_level captures its kernel and
 * memset launches on an internal stream into a CUDA graph and launches the
 * graph on the caller's stream.  The executable graph of each depth is kept
 * per host thread and updated in place (cudaGraphExecUpdate) when the next
 * level step has the same launch structure, so repeated fits of similar
 * trees replay a graph instead of issuing launch by launch.  Results are
 * bitwise the same as without the option. */
#define FMT_OPT_GRAPH 1

typedef struct fmt_tree fmt_tree; /* opaque, device resident */

/* Number of monomials of total degree <= p in 3-D (the rank stride of Sec. 2
 * evaluated at p+1); 0 for p < 0. */
int32_t fmt_nmono(int32_t degree);

/*
 * oct_build -- stage the points and build the root of the octree.
 * Covers the steps before the first Alg. 1 fit: tau = tol_rel * max|f|,
 * residual r := f, the exact quantisation q = floor((x-lo)*2^21/side)
 * clamped to [0, 2^21-1] per axis, 63-bit Morton codes (bit 3j: x bit j,
 * 3j+1: y, 3j+2: z), a stable sort of the points by the top 3*max_depth code
 * bits (every octree node becomes a contiguous range), and the root node.
 *   params   host, read during the call.
 *   n        number of points, n >= 1.
 *   x,y,z,f  device, n doubles each, caller owned (copied into the tree).
 *   out      host; receives the new tree (NULL on failure).
 * Returns FMT_EINVAL for bad parameters or any non-finite input value.
 * Synchronises (reads back max|f| and the input check).
 */
fmt_status oct_build(const fmt_params* params, int64_t n, const double* x, const double* y,
                     const double* z, const double* f, void* stream, fmt_tree** out);

/*
 * fit_level -- Alg. 2 for every active node at `depth`, in parallel.
 * Per node: local frame u = (x - c) * s (Alg. 1 first step), Householder QR
 * of the augmented matrix [Lambda(u) | r] (row chunks reduced pairwise),
 * F = R^{-1} Q^T r with the rank rule (columns with |R_jj| <= 64 nmono eps
 * max|R_kk| are dropped and the rest re-triangularised), the residual update
 * r <- r - Lambda F, and each octant's sum of squared residuals and count.
 * Legal for depth 0 right after oct_build and for depth d+1 after refine(d)
 * reported new nodes; otherwise FMT_EINVAL.  Asynchronous.
 *
 * With precision FMT_MIXED the same least-squares fit is computed another
 * way for nodes of degree <= FMT_MIXED_MAX_DEGREE (the paper has only the
 * FP64 Householder form):
 *  - basis: Legendre products P_a(t_x) P_b(t_y) P_c(t_z), a+b+c <= p, with
 *    t = 2^e u per axis, e >= 0 the largest power of two that keeps the
 *    node's points in |t| <= 1.  It spans the same polynomial space as the
 *    moments of Alg. 2, so the least-squares fit is the same function.
 *  - the Gram matrix [B | r]^T [B | r] of the node (r scaled by a power of
 *    two) is formed on the tensor cores from split-BF16 operands: each value
 *    cut into four fixed-point digits (exact BF16 tiles, pre-scaled), the six
 *    leading digit-tile products accumulated in FP32, promoted to FP64 every
 *    256 rows;
 *  - its FP64 Cholesky factor is the R-hat = [[R, Q^T r], [0, rho]] of the
 *    FP64 path (same matrix, up to row signs); F = R^{-1} Q^T r;
 *  - `sweeps` refinement steps: s = r - Lambda F in FP64, g = B^T s on the
 *    tensor cores as above, F += (R^T R)^{-1} g;
 *  - F is converted exactly to Alg. 2's moment basis in the node frame (the
 *    stored coefficients have the FP64 path's layout), and r <- r - Lambda F
 *    runs in FP64 as on the FP64 path.
 * A node whose root degree was clamped is fitted by the FP64 Householder
 * path, and so are the nodes with fewer than 1.5 m points (m = nmono + 1:
 * nearly square systems, whose Gram is often too ill-conditioned for either
 * normal-equations tier) of a level that has at most 304 items of them:
 * those start at the beginning of the level on a side stream, beside the
 * tensor-core tier (with more, they take the tiers like any other node).  A node whose Cholesky pivot
 * falls below 1e-6 of its diagonal entry (FMT_FLAG_MIXED_PIVOT) is refitted
 * by Householder too.  A node whose fit after the last sweep is not
 * within 1e-7 of converged (the last change |Lambda d|, or its extrapolation
 * by the ratio of the last two changes, above 1e-7 |Lambda F|), or whose
 * polynomial may still change by more than 1e-8 max|f| somewhere in the node
 * box (the same extrapolation of a bound of the last change over the box),
 * or whose polynomial the bias of the quantised basis (|B~ - B| <= 2^-31)
 * may move by more than 1e-8 max|f| over the box (a perturbation of that
 * size solved through R^T R) (FMT_FLAG_MIXED_SLOW), and every node of degree
 * above FMT_MIXED_MAX_DEGREE
 * up to FMT_MIXED_FP64_MAX_DEGREE, goes to the mixed path's FP64 tier: the same basis, its Gram [B|r]^T[B|r]
 * formed in FP64 on the CUDA cores (n m^2 flops, half of Householder's), an
 * FP64 Cholesky (pivot floor 1e-12 of the diagonal), and `sweeps` corrected
 * semi-normal steps with FP64 residuals and FP64 projections under the same
 * convergence tests, plus one more: the change of the polynomial over the
 * box caused by the FP64 rounding of the residual (a perturbation of that
 * size solved through R^T R) must stay within 1e-8 max|f|.  Nodes this tier
 * fits carry FMT_FLAG_MIXED | FMT_FLAG_MIXED_FP64; the rest are refitted by
 * Householder.  Above degree 10 the moment basis of Alg. 2 is so badly scaled
 * (u^14/14! is ~1e-11) that Householder's rank rule drops columns the
 * Legendre basis keeps, so those nodes always take Householder.  Nodes
 * fitted the mixed way carry FMT_FLAG_MIXED.
 * The mixed path targets an interpolant within 1e-6 max|f| of the FP64
 * path (not the 1e-10 of FP64), and its tree may differ where a refinement
 * decision is that close to tau.  FMT_ETIMEOUT if a tensor-core completion
 * wait exceeds 2 s (the tree is then unusable).
 */
fmt_status fit_level(fmt_tree* tree, int32_t depth, void* stream);

/*
 * refine -- the decision loop of Alg. 1 for every node at `depth`:
 * E_RMS = sqrt(S_o / n_o) per octant; octant o becomes a node at depth+1 iff
 * E_RMS > tau, n_o >= max(nmono, min_pts) and depth+1 <= max_depth.  New
 * nodes are compacted in Morton order.  Legal right after fit_level(depth).
 *   n_new_nodes  host, receives the number of nodes created at depth+1.
 * Synchronises (one small device-to-host read).
 */
fmt_status refine(fmt_tree* tree, int32_t depth, int64_t* n_new_nodes, void* stream);

/*
 * oct_build_batch -- oct_build for a forest of independent problems, fitted
 * together level by level (every fit_level / refine covers all problems).
 *   params       host: max_depth, min_pts, tol_rel, precision, chunk_rows
 *                are shared; degree and the box are the defaults.
 *   n_problems   >= 1.
 *   offsets      host, n_problems+1 values, offsets[0] = 0, strictly
 *                increasing: problem i owns inputs offsets[i] .. offsets[i+1]-1.
 *   degrees      host, n_problems values (0..14), or NULL for params->degree.
 *   boxes        host, 4 values per problem (lo x, lo y, lo z, side), or NULL
 *                for params->lo / params->side.
 *   x,y,z,f      device, offsets[n_problems] doubles each, caller owned.
 * tau is per problem: tol_rel * max |f| over that problem's points.  The
 * problem index sits above the Morton bits of the sort key and of the node
 * keys, so ceil(log2(n_problems)) + 3 * (max_depth + 1) must not exceed 64
 * (FMT_EINVAL otherwise).  Synchronises.
 */
fmt_status oct_build_batch(const fmt_params* params, int64_t n_problems, const int64_t* offsets,
                           const int32_t* degrees, const double* boxes, const double* x, const double* y,
                           const double* z, const double* f, void* stream, fmt_tree** out);

/*
 * evaluate -- the tree interpolant at m targets: for each target, the sum
 * over depth d = 0, 1, ... of Lambda(u_d) . F_d for the node at depth d that
 * contains it (same quantisation as oct_build), stopping at the first depth
 * with no such node or past the last fitted level.
 *   xq,yq,zq   device, m doubles each, caller owned.
 *   out        device, m doubles, caller owned, written.
 *   n_outside  host or NULL; if given, receives how many targets lie outside
 *              the closed root cube (they are extrapolated from the clamped
 *              path) and the call synchronises.
 * m = 0 is legal.  Asynchronous unless n_outside is given.
 */
fmt_status evaluate(fmt_tree* tree, int64_t m, const double* xq, const double* yq, const double* zq,
                    double* out, int64_t* n_outside, void* stream);

/*
 * evaluate_batch -- evaluate for a forest: target i is evaluated in the tree
 * of problem target_problem[i] (device, m int32 values in [0, n_problems);
 * may be NULL for a single-problem tree).  An index out of range is reported
 * as FMT_EINVAL when n_outside is given (the call then synchronises).
 */
fmt_status evaluate_batch(fmt_tree* tree, int64_t m, const int32_t* target_problem, const double* xq,
                          const double* yq, const double* zq, double* out, int64_t* n_outside, void* stream);

/* Per-level counters.  Synchronises. */
typedef struct {
  int32_t degree, nmono, max_depth, n_levels; /* n_levels = levels with nodes */
  int32_t n_fitted;                           /* levels whose fit is done */
  int32_t n_problems;
  int64_t n_points;
  double tau, maxabs_f;
  int64_t nodes[FMT_MAX_DEPTH + 1];
  int64_t points[FMT_MAX_DEPTH + 1];
  int64_t items[FMT_MAX_DEPTH + 1];      /* QR work items (row chunks) */
  int64_t chunk_rows[FMT_MAX_DEPTH + 1];
  int64_t near_tau[FMT_MAX_DEPTH + 1];   /* nodes flagged FMT_FLAG_NEAR_TAU */
  int64_t rank_flagged[FMT_MAX_DEPTH + 1];
  int64_t mixed[FMT_MAX_DEPTH + 1];         /* nodes fitted by the mixed path */
  int64_t mixed_points[FMT_MAX_DEPTH + 1];  /* their points */
} fmt_stats;
fmt_status fmt_tree_stats(fmt_tree* tree, fmt_stats* out);

/*
 * Serialised tree ("FMT2" blob, little endian, every array 8-byte aligned).
 * Layout: fmt_export_header, then for the n_nodes nodes (level by level, in
 * node-key order inside a level; a node key is problem << 3*depth | Morton
 * prefix, the prefix being code >> 3*(21-depth)):
 *   uint64 key[n]
 *   int64  start[n]      first point (sorted order)
 *   int64  count[n]      number of points
 *   int32  depth[n], flags[n], deg_used[n], masks[n] (refine_mask | near_mask<<8),
 *          problem[n], pad[n]
 *   double child_E[8n]   RMS residual of each octant after the node's fit
 *   int64  child_n[8n]   points per octant
 *   double coef[nmono*n] F in Alg. 2 order (l outer, m, n inner); nmono of the
 *                        largest degree, zeros past a node's own degree
 * then the problem table (P = n_problems entries):
 *   int32 degree[P], q_root[P] (root degree after the clamp);
 *   double tau[P], maxabs_f[P], lo[3P], side[P]; int64 start[P], count[P]
 * and, when has_points = 1:
 *   uint64 code[N]       full Morton codes, sorted order
 *   int64  perm[N]       sorted position -> input index
 *   double resid[N]      current residual, INPUT order
 * The header's tau, maxabs_f, lo and side are those of problem 0.
 */
typedef struct {
  uint32_t magic;   /* 0x32544d46, "FMT2" */
  uint32_t version; /* 2 */
  int32_t degree, nmono, max_depth, min_pts; /* degree/nmono: the largest */
  int32_t n_levels, n_fitted, has_points, n_problems;
  double tol_rel, tau, maxabs_f, lo[3], side;
  int64_t n_points, n_nodes;
  int64_t level_nodes[FMT_MAX_DEPTH + 1];
} fmt_export_header;

/* Export the tree into host_buf.  With host_buf == NULL only *len is set to
 * the required size.  FMT_EINVAL if *len is too small.  Synchronises. */
fmt_status fmt_tree_export(fmt_tree* tree, void* host_buf, size_t* len);

/* Rebuild an evaluation-only tree from a blob (has_points may be 0; every
 * level in the blob is taken as fitted).  fit_level/refine on it return
 * FMT_EINVAL.  Synchronises.  host_buf (len bytes) is the caller's and is
 * only read.  Before any device work the whole blob is checked on the host:
 * header fields, every count against the bytes present (so no count can
 * overflow the size check), each problem's degree and box, each node's
 * problem index, and each level's strictly increasing node keys.  A
 * truncated or inconsistent blob returns FMT_EINVAL and allocates nothing;
 * *out is NULL on every error. */
fmt_status fmt_tree_import(const void* host_buf, size_t len, void* stream, fmt_tree** out);

/*
 * Kernel-level instrumentation (no counterpart in the paper; it serves the
 * roofline measurements).  Process-wide counters per kernel class: number of
 * kernel launches, and -- while enabled -- the device time between CUDA events
 * recorded on the launching stream right before and after each launch, plus
 * the work units the launch processed (rows for tile_qr/residual, node pairs
 * for combine, nodes for back_solve/refine, targets x fitted levels for
 * evaluate, points for the build kernels).  tile_qr counts one launch per
 * degree present in the level.  The class "graph_launch" counts the graphs
 * launched under FMT_OPT_GRAPH (units: those that reused an executable graph
 * updated in place); the kernels inside are counted in their own classes, and
 * their events are recorded inside the graph.  The mixed path's classes are
 * mixed_* (tensor-core tier) and fp64_* (its FP64 normal-equations tier).
 * fmt_profile_enable(1) resets the counters and starts event timing;
 * fmt_profile_enable(0) stops it.  fmt_profile_read synchronises the device.
 */
#define FMT_PROFILE_CLASSES 24
typedef struct {
  int64_t launches[FMT_PROFILE_CLASSES];
  double ms[FMT_PROFILE_CLASSES];
  double units[FMT_PROFILE_CLASSES];
  double flops[FMT_PROFILE_CLASSES]; /* algorithmic FP64 flops (FMA = 2) */
} fmt_profile;
fmt_status fmt_profile_enable(int32_t on);
fmt_status fmt_profile_read(fmt_profile* out);
/* Name of a kernel class ("tile_qr", ...), or NULL past the last class. */
const char* fmt_profile_class_name(int32_t k);

/*
 * FP64 pipe throughput probe (no counterpart in the paper): runs a kernel of
 * independent fused multiply-adds on every SM for about `iters` x 8 DFMA per
 * thread and returns the measured rate in DFMA per second (FLOP/s = 2x).  It
 * is the denominator of the FP64 roofline reported next to the fit kernels.
 * Synchronises.
 */
fmt_status fmt_probe_dfma(int64_t iters, double* dfma_per_s, void* stream);

/*
 * Autotuner of the FP64 Householder fit (no counterpart in the paper, which
 * fixes no GPU schedule).  For each degree p the library keeps one launch
 * configuration of the QR of fit_level (Alg. 2 per node, chunks reduced
 * pairwise):
 *   rows          rows of [Lambda | r] absorbed per shared-memory block:
 *                 16, 32, 48, 64 or 128, and (rows + 2) * ld * 8 + 32 bytes must fit
 *                 in 227 KB, ld = the padded row pitch of nmono(p) + 1 columns;
 *   warps         warps per tile-QR CTA: 4 or 8;
 *   chunk_factor  smallest row chunk (one work item of the persistent queue)
 *                 = chunk_factor * (nmono + 1) rows rounded up to 64:
 *                 1, 2, 4, 8 or 16 (fmt_params.chunk_rows > 0 overrides it;
 *                 a forest of several degrees keeps the built-in 4);
 *   merge         pairwise reduction of a node's chunk triangles: 0 packs the
 *                 second triangle into shared memory where it fits (nmono+1
 *                 <= 166), 1 always streams it in row blocks.
 * A degree without a tuned or installed entry uses the built-in rule
 * (source 0): the largest of 64/32/16 rows that fits two (64) or one CTA per
 * SM, 4 warps (8 from degree 8 on), chunk_factor 4, merge 0.  The configuration changes the order
 * of floating-point operations, not the method: every configuration meets
 * the same accuracy, and runs with one table are bitwise reproducible.  The
 * tile QR of a level runs one launch per degree present (on side streams,
 * largest degree first), each with its degree's entry; the merges use the
 * entry of the level's largest degree.  The table
 * is per process (all devices of this pool are alike); change it only while
 * no fit is running.
 *
 * fmt_autotune times candidate configurations for `degree` on a synthetic
 * forest of `sample_points` uniform random points (0 selects a size that
 * keeps one trial near 50 ms): half in one problem, half in equal problems of
 * at least 8 (nmono + 1) points each, tau = 0, depth 0, so that both one big
 * node spread over every SM and many small nodes are in the timed work.  It
 * times fit_level(0) with CUDA events (best of two after a warm-up) and
 * searches coordinate-wise: rows x warps, then chunk_factor, then merge.
 * The winner is installed (source 1) and returned in *out with its time and
 * the time of the built-in rule on the same sample.  Synchronises; allocates
 * and frees its own device memory.  FMT_EINVAL for a degree outside 0..14.
 *
 * fmt_tune_get returns the entry in force for `degree` (host only, no GPU
 * needed).  fmt_tune_set installs an entry (e.g. one saved from an earlier
 * autotune) after checking the values above, or with source = 0 restores the
 * built-in rule for that degree; FMT_EINVAL on a bad value.
 */
typedef struct {
  int32_t degree;
  int32_t rows;
  int32_t warps;
  int32_t chunk_factor;
  int32_t merge;
  int32_t source;        /* 0 built-in rule, 1 autotuned, 2 installed by fmt_tune_set */
  int64_t sample_points; /* autotune: points timed per trial */
  double ms;             /* autotune: fit_level(0) time of this configuration */
  double ms_builtin;     /* autotune: fit_level(0) time of the built-in rule */
  int32_t trials;        /* autotune: configurations timed */
  int32_t pad;
} fmt_tune_entry;
fmt_status fmt_autotune(int32_t degree, int64_t sample_points, void* stream, fmt_tune_entry* out);

/*
 * fmt_autotune_forest -- the autotuner on the forest a caller is about to
 * fit (no counterpart in the paper).  A one-degree trial cannot see how the
 * per-degree tile-QR launches of a level share the GPU, so this one times
 * the whole level loop (fit_level / refine to the end, after
 * oct_build_batch) of the given problems -- a sample of the real forest,
 * e.g. its first few hundred problems -- with the table in force, then
 * degree by degree (every degree present, largest first) the candidates
 * warps 4 <-> 8 and rows 32 / 64 / 128 where they fit, each timed on the
 * same forest, keeping a candidate when the whole loop is more than 2%
 * faster than the incumbent.  The winners stay installed (source 1);
 * chunk_factor and merge are left as they are.
 *   params .. f   as for oct_build_batch (device point arrays).
 *   report        host or NULL: time of the loop with the table at entry
 *                 (ms_start) and with the result (ms_best), trials, and the
 *                 number of entries changed.
 * Synchronises; allocates through the trees it builds and frees them.  On
 * an error the table at entry is restored.
 */
typedef struct {
  double ms_start, ms_best;
  int32_t trials, changed;
} fmt_tune_report;
fmt_status fmt_autotune_forest(const fmt_params* params, int64_t n_problems, const int64_t* offsets,
                               const int32_t* degrees, const double* boxes, const double* x, const double* y,
                               const double* z, const double* f, void* stream, fmt_tune_report* report);
fmt_status fmt_tune_get(int32_t degree, fmt_tune_entry* out);
fmt_status fmt_tune_set(const fmt_tune_entry* entry);

/*
 * Failure-path diagnostics (no counterpart in the paper).
 * fmt_debug_fail_alloc(k): the k-th device allocation the library makes from
 * now on (k >= 1) fails as if the device were out of memory: the call that
 * needed it returns FMT_ENOMEM and the tree stays safe to free; k = 0
 * disarms.  Process-wide; host only (no GPU needed).  FMT_EINVAL for k < 0.
 * fmt_wait_probe(limit_ns): one thread waits on an mbarrier that nothing
 * arrives on, through the same bounded wait the mixed kernels use for their
 * tensor-core completions (bound 2 s there), here with the bound limit_ns
 * (1e3..1e10 ns).  It returns FMT_ETIMEOUT when the bound runs out -- the
 * error path of a stuck completion -- and the context stays usable: no trap,
 * no hang.  Synchronises.  FMT_EINVAL for a bound outside the range.
 */
fmt_status fmt_debug_fail_alloc(int64_t k);
fmt_status fmt_wait_probe(int64_t limit_ns, void* stream);

/*
 * Bounds-checked build.  Compiled with -DFMT_CHECKED, every kernel tests the
 * indices it reads from device memory (a work item's node, rows and scratch
 * slot; a node's problem, points, items and coefficient slot; a parent found
 * by search; a sort position) against the sizes of the buffers it addresses,
 * before any access through them.  A failed test skips the guarded work and
 * records where it failed; oct_build, oct_build_batch, fit_level, refine,
 * evaluate(_batch), fmt_tree_import and fmt_fit_node_static then synchronise
 * the device and return FMT_EINTERNAL, fmt_last_error naming the first failed
 * site.  (While the stream is being captured into a graph nothing has run
 * yet, and nothing is read.)  The default build compiles the tests out.
 * fmt_checked_build(): 1 for the checked build, else 0.
 * fmt_check_probe(i, n): the mechanism's self-test.  One thread writes
 * element i (0 <= i < 64) of a 64-element device array when the checked
 * build's test i < n (0 <= n <= 32) passes; the default build writes it
 * unconditionally (always inside the array).  The checked build returns
 * FMT_EINTERNAL for i >= n, else FMT_OK; the default build FMT_OK.
 * Synchronises.  FMT_EINVAL for i or n outside those ranges.
 * fmt_debug_item_rows(tree, depth, item, start, end): test hook that sets
 * the row range of one work item of a planned, not yet fitted level, with
 * 0 <= start <= end <= n (FMT_EINVAL otherwise), so that every access stays
 * inside the point arrays; a range outside the item's node is what the
 * checked build's tests report at the next fit_level.
 */
int32_t fmt_checked_build(void);
fmt_status fmt_check_probe(int32_t i, int32_t n, void* stream);
fmt_status fmt_debug_item_rows(fmt_tree* tree, int32_t depth, int64_t item, int64_t start, int64_t end,
                               void* stream);

/*
 * fmt_fit_node_static -- allocation-free least-squares fit of ONE point set.
 * The paper has no counterpart: this exists for callers that cannot let a
 * library allocate device memory -- code whose device memory is owned by
 * another allocator or a fixed budget, or that must not risk the implicit
 * device synchronisation and run-time out-of-memory failures of cudaMalloc.
 * It performs the per-node fit of the tree path (Householder QR of
 * [Lambda(u) | r], back substitution with the rank rule, residual update) for
 * a single node whose box is the root cube [lo, lo+side)^3, and allocates
 * nothing: its scratch is one static device array of 166 x 166 doubles
 * (220,448 bytes, FMT_STATIC_MAX_DEGREE = 8), which stays on every GPU that
 * loads the library until the process exits.
 *   degree   0 <= degree <= FMT_STATIC_MAX_DEGREE, else FMT_EINVAL with a
 *            message naming the limit.  When n < nmono(degree) the degree is
 *            lowered as at the root of a tree (flag FMT_FLAG_DEG_CLAMPED).
 *   n        number of points, 1 <= n < 2^31.
 *   x,y,z    device, n doubles each (global coordinates), caller owned.
 *   r_in     device, n doubles: the values to fit, caller owned.
 *   lo, side host: the box, read during the call.
 *   coef     device, nmono(degree) doubles, written: the coefficients of the
 *            monomials u^l v^m w^n / (l! m! n!), l outermost, then m, then n
 *            innermost (the coef layout of fmt_tree_export); with a lowered
 *            degree the coefficients of the dropped monomials are zero.
 *   r_out    device, n doubles, written: r_in - Lambda F (may equal r_in).
 *   flags    device int32 or NULL, written: FMT_FLAG_RANK | FMT_FLAG_DEG_CLAMPED.
 * One CTA does the whole fit, so it suits small point sets (it is slow for
 * millions of points).  Every call on a device uses the same scratch array
 * and leaves its contents behind (each call clears what it reads before
 * use): calls that can overlap on the GPU (different streams, or threads
 * without ordering) race and corrupt each other -- order them on one stream.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it with the id of the device's context;
 * make that first call before any stream capture.  A call that finds a
 * different context (after cudaDeviceReset the module is reloaded at a new
 * address) looks the address up again.  Asynchronous.
 */
#define FMT_STATIC_MAX_DEGREE 8
fmt_status fmt_fit_node_static(int32_t degree, int64_t n, const double* x, const double* y, const double* z,
                               const double* r_in, const double* lo, double side, double* coef, double* r_out,
                               int32_t* flags, void* stream);

/* Release the tree (waits for its last stream).  NULL is ignored. */
void fmt_tree_free(fmt_tree* tree);

/* Free the scratch only fitting uses (the QR triangles of the work items and
 * the mixed path's Gram, projection, sweep-residual and digit-tile buffers),
 * stream-ordered on `stream`, for a tree kept for evaluation (no
 * counterpart in the paper).  Evaluation, stats and export are unaffected;
 * a later fit_level allocates the scratch again.  FMT_EINVAL for NULL. */
fmt_status fmt_tree_trim(fmt_tree* tree, void* stream);

/* Message of the last failure on `tree`, or of the calling thread's last
 * failure when tree == NULL (e.g. a failed oct_build).  Never NULL. */
const char* fmt_last_error(const fmt_tree* tree);

/*
 * Serving (no counterpart in the paper; every numerical step is the calls
 * above).  Fit+evaluate requests are queued and run by `slots` worker
 * threads, each with its own CUDA stream.  A slot that frees up forms its
 * next batch from the oldest queued request and every queued request with
 * the same batch key (params.precision, max_depth, min_pts, tol_rel, sweeps,
 * chunk_rows), as long as the batch stays within max_batch_points (the first
 * request always goes) and the sum of the admitted requests' device-memory
 * estimates stays within budget_bytes; the batch runs as one forest
 * (oct_build_batch with each request's degree and box, the fit_level/refine
 * loop, evaluate_batch).  So requests that arrive while other batches are on
 * the GPU join the next batch, and batches of different slots overlap on the
 * device.  A request whose estimate alone exceeds the budget completes with
 * FMT_ENOMEM.  Each request's tree is independent of the others in its
 * batch; its result equals the result of running it alone up to the
 * rounding of a different row-chunk plan (FP64: within 1e-10 max|f|).
 *
 * The batch key also holds the request's size class (the decade of its
 * point count), so a batch of small requests does not wait for a large one.
 *
 *   fmt_request   params: the request's fmt_params (degree, lo, side are per
 *                 request; the rest is the batch key).  x,y,z,f: host, n
 *                 each; xq,yq,zq: host, m each; out: host, m.  All must stay
 *                 valid and unmodified until fmt_server_wait returns it.
 *                 keep: 1 keeps the request's tree (the forest of its batch)
 *                 resident on the device after the batch; 0 frees it.
 *   fmt_request_result  status of the request; t_submit / t_start / t_done
 *                 on fmt_server_clock(); the batch it ran in; with keep, the
 *                 id of the resident tree (resident_id > 0) and the
 *                 request's problem index in it.
 * Resident trees: fmt_server_submit_eval queues an evaluate-only request
 * (host targets xq, yq, zq and output out, m each, valid until the wait)
 * against a resident tree, run by the next free slot; it evaluates the
 * kept request's own tree, so it gives what the fit's own evaluation gave
 * at the same targets.  fmt_server_release drops a resident tree (after
 * evaluations already queued on it); a forest is freed when the last of its
 * kept requests is released.  A kept forest's fit scratch is freed at once
 * (fmt_tree_trim); its resident estimate (about 400 bytes per point) stays
 * counted against budget_bytes until the release.  FMT_EINVAL for an unknown
 * or released id.  fmt_server_memory reports the bytes currently admitted
 * (running batches and resident forests), their peak, and the number of
 * resident trees; staging buffers are pool allocations freed with their
 * batch, so device use stays within what was admitted.
 * fmt_server_create: slots 1..64, budget_bytes > 0, max_batch_points >= 1;
 *   uses the current device.  fmt_server_submit copies the request struct
 *   (not the arrays) and returns a ticket; FMT_EINVAL for bad fields.
 * fmt_server_wait: blocks until the request is done (timeout_s < 0: no
 *   limit; FMT_ETIMEOUT otherwise) and releases the ticket.
 * fmt_server_destroy: runs what is queued, joins the slots, frees.
 */
typedef struct fmt_server fmt_server;
typedef struct {
  fmt_params params;
  int64_t n, m;
  const double *x, *y, *z, *f;
  const double *xq, *yq, *zq;
  double* out;
  int32_t keep;
  int32_t pad;
} fmt_request;
typedef struct {
  fmt_status status;
  int32_t batch_requests;
  int64_t batch_id, batch_points;
  double t_submit, t_start, t_done;
  int64_t resident_id;
  int32_t problem;
  int32_t pad;
} fmt_request_result;
fmt_status fmt_server_create(int32_t slots, double budget_bytes, int64_t max_batch_points, fmt_server** out);
fmt_status fmt_server_submit(fmt_server* server, const fmt_request* request, int64_t* ticket);
fmt_status fmt_server_wait(fmt_server* server, int64_t ticket, double timeout_s, fmt_request_result* result);
fmt_status fmt_server_destroy(fmt_server* server);
fmt_status fmt_server_submit_eval(fmt_server* server, int64_t resident_id, int64_t m, const double* xq,
                                  const double* yq, const double* zq, double* out, int64_t* ticket);
fmt_status fmt_server_release(fmt_server* server, int64_t resident_id);
fmt_status fmt_server_memory(fmt_server* server, double* admitted, double* peak_admitted, int64_t* resident_trees);
double fmt_server_clock(void); /* seconds, steady clock of the server */

#ifdef __cplusplus
}
#endif
#endif /* FMT_H */
