// fmt_internal.cuh -- internal types and device helpers of libfmt (not part of
// the C ABI).  Every kernel is declared here through a host launcher (build,
// FP64 fit, mixed path and its FP64 tier, refine and evaluation, the DFMA
// and bounded-wait probes), with the per-degree QR launch-configuration
// table; fmt_api.cu sequences them.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fmt.h"

#define FMT_QBITS 21
#define FMT_STATIC_MAX_M 166  // nmono(FMT_STATIC_MAX_DEGREE) + 1
#define FMT_QMAX 0x1fffffu

// device error word bits
#define FMT_ERR_NONFINITE 1
#define FMT_ERR_INDEX 2
#define FMT_ERR_CAPACITY 4
#define FMT_ERR_TIMEOUT 8

// ---------------------------------------------------------------------------
// Bounds-checked build (nvcc -DFMT_CHECKED).  Before a kernel addresses
// memory through an index it read from device memory (a work item's node,
// rows and scratch slot, a node's problem, points, items and coefficient
// slot, a parent found by search), it tests that index against the size of
// the buffer it addresses.  A failed test records its site in the check word
// of its translation unit and skips the work it guards, so no access leaves
// its buffer; the results are then incomplete, and the ABI call that
// launched the kernel synchronises, reads every check word and returns
// FMT_EINTERNAL naming the first failed site.  In the default build
// FMT_CHECK(cond, site) is the constant true and cond is not evaluated.
// The tests are uniform over a CTA (a cluster, for the cluster merge), so
// skipping never splits a barrier.
enum fmt_check_site {
  CK_NONE = 0,
  CK_BUILD_INDEX,    // build: a point's problem, a sort position or a permutation entry
  CK_PLAN_NODE,      // plan: a node's problem, degree or point range
  CK_QR_ITEM,        // tile QR: the item, its node, rows, problem or R triangle
  CK_MERGE_ITEM,     // merges: the pair of items and their R triangles
  CK_BACKSOLVE_NODE, // back substitution: the node's R triangle or coefficient slot
  CK_RESIDUAL_ITEM,  // residual update: the item, its node and rows
  CK_CHILD_NODE,     // child statistics: a node's points or octant bounds
  CK_MIXED_ITEM,     // mixed path, per item: node, rows, accumulator slot
  CK_MIXED_NODE,     // mixed path, per node: its items, problem and scratch
  CK_EVAL_NODE,      // evaluation: a node's problem or coefficient slot
  CK_CUM_NODE,       // cumulative polynomials: a node, its problem or parent
  CK_STATIC_ROWS,    // allocation-free fit: the rows or the degree
  CK_PROBE,          // fmt_check_probe: the self-test of the mechanism
  CK_SITES
};

// Sizes a level's indices are tested against (every build passes them; only
// the checked build reads them).
struct fmt_bounds {
  int64_t n_points;   // sorted points of the tree
  int64_t n_nodes;    // nodes of the level
  int64_t n_items;    // work items of the level
  int64_t r_cap;      // doubles of QR scratch the level's triangles may use
  int32_t n_problems; // entries of the problem table
  int32_t max_m;      // largest m (nmono + 1) a node of the level may have
};

__host__ __device__ __forceinline__ bool fmt_in(int64_t i, int64_t n) { return i >= 0 && i < n; }

#ifdef FMT_CHECKED
static __device__ int g_fmt_check_site;  // this translation unit's first failed site
__device__ __forceinline__ bool fmt_check_fail(int site) {
  atomicCAS(&g_fmt_check_site, 0, site);
  return false;
}
#define FMT_CHECK(cond, site) ((cond) || fmt_check_fail(site))
// defines fn(): this translation unit's failed site (0: none), then clears it
#define FMT_CHECK_READER(fn)                                              \
  int fn() {                                                              \
    int v = 0;                                                            \
    if (cudaMemcpyFromSymbol(&v, g_fmt_check_site, sizeof v) != cudaSuccess) return -1; \
    if (v != 0) {                                                         \
      const int zero = 0;                                                 \
      cudaMemcpyToSymbol(g_fmt_check_site, &zero, sizeof zero);           \
    }                                                                     \
    return v;                                                             \
  }
int check_site_build();
int check_site_fit();
int check_site_mixed();
int check_site_plan();
#else
#define FMT_CHECK(cond, site) true
#endif
const char* check_site_name(int site);

// 1/l! for l = 0..14, each a correctly rounded binary64 quotient (l! is exact)
static __constant__ double c_invfact[FMT_MAX_DEGREE + 1] = {
    1.0,          1.0,          1.0 / 2.0,          1.0 / 6.0,           1.0 / 24.0,
    1.0 / 120.0,  1.0 / 720.0,  1.0 / 5040.0,       1.0 / 40320.0,       1.0 / 362880.0,
    1.0 / 3628800.0, 1.0 / 39916800.0, 1.0 / 479001600.0, 1.0 / 6227020800.0, 1.0 / 87178291200.0};

// ---------------------------------------------------------------------------
// Morton codes: 21 bits per axis; bit 3j <- x bit j, 3j+1 <- y, 3j+2 <- z.
__host__ __device__ inline uint64_t fmt_spread3(uint64_t v) {
  v &= 0x1fffffull;
  v = (v | (v << 32)) & 0x1f00000000ffffull;
  v = (v | (v << 16)) & 0x1f0000ff0000ffull;
  v = (v | (v << 8)) & 0x100f00f00f00f00full;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}
__host__ __device__ inline uint32_t fmt_compact3(uint64_t v) {
  v &= 0x1249249249249249ull;
  v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
  v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
  v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
  v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
  v = (v ^ (v >> 32)) & 0x1fffffull;
  return (uint32_t)v;
}

// Exact quantisation: floor((x - lo) * S), S = 2^21/side, clamped; the
// subtraction and the product are separately rounded (no contraction).  The
// floor is one conversion to a 64-bit integer, which saturates (and sends a
// NaN below zero), clamped with integer compares.
__device__ __forceinline__ int64_t fmt_floor_scaled(double x, double lo, double S) {
  return __double2ll_rd(__dmul_rn(__dsub_rn(x, lo), S));
}
__device__ __forceinline__ uint32_t fmt_clamp_q(int64_t f) {
  return f < 0 ? 0u : (f > (int64_t)FMT_QMAX ? FMT_QMAX : (uint32_t)f);
}
__device__ __forceinline__ uint32_t fmt_quant(double x, double lo, double S) {
  return fmt_clamp_q(fmt_floor_scaled(x, lo, S));
}

// Node frame of Alg. 1: h = side 2^-(d+1), c = lo + (2i+1) h, s = 1/h.
// inv_side = 1/side rounded once on the host: h is side times a power of two,
// so 1/h rounded is exactly inv_side 2^(d+1) (scaling by a power of two
// commutes with rounding), which spares every frame a division.
__device__ __forceinline__ void fmt_frame(double lo, double side, double inv_side, int depth, uint32_t i,
                                          double& c, double& s) {
  double h = ldexp(side, -(depth + 1));
  c = __dadd_rn(lo, __dmul_rn((double)(2u * i + 1u), h));
  s = ldexp(inv_side, depth + 1);
}

// u = (x - c) * s without contraction
__device__ __forceinline__ double fmt_local(double x, double c, double s) {
  return __dmul_rn(__dsub_rn(x, c), s);
}

// Polynomial of a node in Horner form.  G holds F_lmn / (l! m! n!) in Alg. 2
// order (l outer, m, n inner, all ascending); reading it backwards visits
// (l, m, n) in descending lexicographic order, which is exactly the nested
// Horner order  sum_l u^l sum_m v^m sum_n w^n G_lmn.
// kGlobal: G is in global memory and read through the read-only path
// (ld.global.nc, global addresses only); otherwise plain generic loads.
template <bool kGlobal>
__device__ __forceinline__ double fmt_horner_t(const double* __restrict__ G, int p, int nmono, double u,
                                               double v, double w) {
  int idx = nmono - 1;
  double P = 0.0;
  for (int l = p; l >= 0; --l) {
    double t = 0.0;
    for (int m = p - l; m >= 0; --m) {
      double s = 0.0;
      for (int n = p - l - m; n >= 0; --n) s = fma(s, w, kGlobal ? __ldg(G + idx--) : G[idx--]);
      t = fma(t, v, s);
    }
    P = fma(P, u, t);
  }
  return P;
}
__device__ __forceinline__ double fmt_horner(const double* __restrict__ G, int p, int nmono, double u, double v,
                                             double w) {
  return fmt_horner_t<true>(G, p, nmono, u, v, w);
}

// double-float arithmetic (Dekker / Knuth error-free transformations)
struct dfl {  // value h + l, |l| <= ulp(h) / 2
  float h, l;
};
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
  const float p = __fmul_rn(x.h, y.h);
  float e = __fmaf_rn(x.h, y.h, -p);
  e = __fmaf_rn(x.h, y.l, e);
  e = __fmaf_rn(x.l, y.h, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ dfl df_sub(dfl x, dfl y) {
  const float s = __fsub_rn(x.h, y.h);
  const float bb = __fsub_rn(s, x.h);
  const float e = __fadd_rn(__fsub_rn(x.h, __fsub_rn(s, bb)), __fsub_rn(-y.h, bb));
  return fast_two_sum(s, __fadd_rn(e, __fsub_rn(x.l, y.l)));
}
__device__ __forceinline__ dfl df_of(double v) {
  const float h = __double2float_rn(v);
  return {h, __double2float_rn(v - (double)h)};
}
__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
  const float s = __fadd_rn(x.h, y.h);
  const float bb = __fsub_rn(s, x.h);
  const float e = __fadd_rn(__fsub_rn(x.h, __fsub_rn(s, bb)), __fsub_rn(y.h, bb));
  return fast_two_sum(s, __fadd_rn(e, __fadd_rn(x.l, y.l)));
}
// x * w + c in double-float
__device__ __forceinline__ dfl df_fma(dfl x, dfl w, dfl c) { return df_add(df_mul(x, w), c); }

// The node polynomial of fmt_horner_t in double-float: the same nested Horner
// order, with the coefficients as (hi, lo) pairs stored in the order Horner
// reads them (Gr[k] = G[nmono - 1 - k]) from a 16-byte boundary, so that one
// 16-byte load brings two of them (the evaluation is bound by the number of
// L1 sectors it reads: one coefficient per load, a target per thread, the
// threads of a warp on different nodes).
__device__ __forceinline__ int fmt_df_stride(int stride) { return (stride + 1) & ~1; }
__device__ __forceinline__ dfl fmt_horner_df(const float2* __restrict__ Gr, int p, dfl u, dfl v, dfl w) {
  const float4* G4 = reinterpret_cast<const float4*>(Gr);
  int k = 0;
  float4 pair = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  dfl P = {0.0f, 0.0f};
  for (int l = p; l >= 0; --l) {
    dfl t = {0.0f, 0.0f};
    for (int m = p - l; m >= 0; --m) {
      dfl s = {0.0f, 0.0f};
      for (int n = p - l - m; n >= 0; --n, ++k) {
        if (!(k & 1)) pair = __ldg(G4 + (k >> 1));
        const dfl g = (k & 1) ? dfl{pair.z, pair.w} : dfl{pair.x, pair.y};
        s = df_fma(s, w, g);
      }
      t = df_fma(t, v, s);
    }
    P = df_fma(P, u, t);
  }
  return P;
}

// nmono(p) on the device
__host__ __device__ __forceinline__ int fmt_nmono_d(int p) { return p < 0 ? 0 : (p + 1) * (p + 2) * (p + 3) / 6; }

// Mixed path: a node with fewer than 1.5 m points (m = nmono + 1) is nearly
// square, its Gram often too ill-conditioned for both normal-equations tiers;
// on a level with few such nodes (route_hard) they go straight to
// Householder, refitted at the start of the level beside the tensor-core tier.
__host__ __device__ __forceinline__ bool fmt_mixed_hard(int degree, int64_t count) {
  return 2 * count < 3 * (int64_t)(fmt_nmono_d(degree) + 1);
}

// Shared-memory row pitch of the QR kernels for m columns: the smallest
// ld >= m with ld = 4 (mod 16) doubles (64-bit accesses are served per
// half-warp: 4 columns x 4 row groups; this puts the row groups of a quad
// pattern in distinct 32-byte bank segments).
__host__ __device__ __forceinline__ int fmt_ld_for(int m) { return m + ((4 - m) & 15); }

// ---------------------------------------------------------------------------
// A forest holds independent problems; every problem has its own root box,
// degree and threshold.  Point ranges are in sorted order (problems keep the
// input order, so these are also the input ranges).
struct fmt_problem {
  double lo[3];
  double side;
  double S;       // 2^21 / side
  double tau;     // tol_rel * max |f| over the problem's points
  double maxabs;
  int32_t degree; // p
  int32_t q_root; // root degree after the N < nmono clamp
  int64_t start, count;
  double inv_side;  // 1 / side (fmt_frame)
  double hi[3];     // lo + side, rounded once (the cube's upper faces)
};

// Node keys of a forest: the problem id sits above the 3d Morton bits of a
// node at depth d, so one sorted array per level covers every problem.
__host__ __device__ __forceinline__ uint64_t fmt_morton_part(uint64_t key, int depth) {
  return depth == 0 ? 0ull : (key & ((1ull << (3 * depth)) - 1ull));
}
__host__ __device__ __forceinline__ int fmt_problem_of(uint64_t key, int depth) {
  return (int)(key >> (3 * depth));
}

// ---------------------------------------------------------------------------
// One octree level as stored on the device (structure of arrays).
struct fmt_level {
  // host-side copies of the sizes
  int64_t n_nodes = 0, cap_nodes = 0;
  int64_t n_items = 0, cap_items = 0, max_chunks = 0, chunk_rows = 0, n_points = 0;
  int32_t max_m = 0;  // largest nmono + 1 among this level's nodes
  int64_t deg_mask = 0;  // degrees present among this level's nodes (bit q)
  double qr_flops = 0.0, horner_flops = 0.0;  // algorithmic flops of the level's fit
  bool fitted = false;
  // nodes
  uint64_t* prefix = nullptr;  // (problem << 3d) | Morton prefix (code >> 3(21-d))
  int32_t* prob = nullptr;     // problem of the node
  int64_t* start = nullptr;
  int64_t* count = nullptr;
  int32_t* flags = nullptr;
  int32_t* deg_used = nullptr;
  int32_t* masks = nullptr;    // refine_mask | near_mask << 8
  int64_t* bounds = nullptr;   // 9 per node: octant ranges in sorted order
  double* child_S = nullptr;   // 8 per node: sum of squared residuals
  int64_t* child_n = nullptr;  // 8 per node
  double* child_E = nullptr;   // 8 per node: RMS
  double* coef = nullptr;      // nmono per node: F (Alg. 2 order)
  double* hcoef = nullptr;     // nmono per node: F / (l! m! n!) for Horner
  double* frame = nullptr;     // 6 per node: c, s of x, y, z (fmt_frame), for evaluation
  double* ccoef = nullptr;     // nmono per node: the node's and all its ancestors' polynomials summed,
                               // as one polynomial in the node's frame (Horner form, like hcoef)
  float2* ccoef_df = nullptr;  // mixed trees: ccoef as double-float (hi, lo) for evaluation
  int64_t* node_item0 = nullptr;
  int32_t* node_nitems = nullptr;
  // QR work items: (node, [start, end)) row chunks, node-major
  int64_t* item_node = nullptr;
  int64_t* item_start = nullptr;
  int64_t* item_end = nullptr;
  int32_t* item_local = nullptr;  // chunk index inside its node
  int32_t* sched = nullptr;       // item order for the QR queue (largest first)
  int64_t* item_roff = nullptr;   // offset of the item's m x m triangle in the QR scratch
  int64_t r_total = 0;            // doubles of QR scratch the level needs
  int64_t n_hard_items = 0;       // items of the mixed path's nearly square nodes (fmt_mixed_hard)
};

// Small result block that refine reads back in one copy.
// work-queue counters per tree: slot 0 for single launches, slot 1 + q for
// the tile-QR launch of degree q
// d_work slots: 0 the mixed Gram's queue; 1 + q the tile QR's; 16 + q the
// early refits'; kPivSlot the tensor-core tier's small-pivot count of a level
constexpr int kPivSlot = 2 * (FMT_MAX_DEGREE + 1) + 1;
constexpr int kWorkSlots = kPivSlot + 1;
// a level refits its small-pivot nodes early (beside the sweeps) only when
// there are at most this many: more Householder work than that competes with
// the sweeps for the SMs
constexpr int kEarlyRefitMax = 64;

struct fmt_plan_out {
  int64_t n_new, n_items, max_chunks, chunk_rows, n_points, n_near, err;
  int64_t max_m;       // largest nmono + 1 among the planned nodes
  double qr_flops;     // sum over nodes of rows x 2 m^2 (Householder on [Lambda | r])
  double horner_flops; // sum over nodes of rows x Horner flops of the node degree
  int64_t r_total;     // doubles of QR scratch: sum over items of m^2
  int64_t deg_mask;    // bit q set: some planned node has (effective) degree q
  int64_t n_hard_items; // items of nodes the mixed path sends straight to Householder
};

// Scratch of the mixed-precision fit (fmt_mixed.cu), grown per tree.
struct fmt_mixed_bufs {
  double* s = nullptr;                  // n: sweep residual
  unsigned long long* mstat = nullptr;  // 8 per node
  double* acc = nullptr;                // acc_stride per item
  int64_t acc_stride = 0;
  double* gacc = nullptr;               // 256 per item
  double* dproj = nullptr;              // FP64 tier: nmono per item (B^T s)
  double* lcoef = nullptr;              // nmono per node
  uint8_t* cache = nullptr;             // digit tiles of the projection basis, or NULL
  size_t cap_cache = 0;
  int64_t cap_nodes = 0, cap_items = 0, cap_acc = 0, cap_dproj = 0;
};

struct fmt_tree {
  fmt_params P{};   // shared parameters (degree and box of problem 0 when P == 1)
  int32_t nmono = 0;       // coefficient stride: nmono of the largest degree
  int32_t max_degree = 0;
  int64_t n = 0;
  int64_t n_problems = 1;
  bool imported = false;
  int device = 0;
  cudaStream_t stream = nullptr;  // last stream used (for the final free)
  // the tile QR's per-degree launches run on side streams forked from the
  // caller's (created on first use, destroyed with the tree)
  cudaStream_t side[FMT_MAX_DEGREE + 1] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[FMT_MAX_DEGREE + 1] = {};
  // mixed path: the Householder refits of small-pivot nodes run on piv_stream
  // while the sweeps run on the caller's stream
  cudaStream_t piv_stream = nullptr;
  cudaEvent_t piv_fork = nullptr, piv_join = nullptr;
  bool piv_pending = false;
  double tau = 0.0, maxabs = 0.0; // problem 0 (single-problem trees)
  int sort_bits = 0;       // Morton bits in the sort key (3 per sorted level)
  int pid_bits = 0;        // problem-id bits above them
  fmt_problem* d_prob = nullptr;  // device table
  fmt_problem* h_prob = nullptr;  // host copy
  // sorted point data
  double *x = nullptr, *y = nullptr, *z = nullptr, *r = nullptr;
  uint64_t* code = nullptr;
  uint32_t* perm = nullptr;
  // levels
  fmt_level lv[FMT_MAX_DEPTH + 1];
  int32_t n_levels = 0;     // levels that hold nodes
  int32_t next_fit = 0;     // depth fit_level expects next
  int32_t next_refine = -1; // depth refine expects next
  int32_t done = 0;         // no further levels
  // scratch
  double* Rbuf = nullptr;
  size_t Rbuf_cap = 0;  // doubles
  int* d_err = nullptr;
  fmt_plan_out* d_plan = nullptr;
  fmt_plan_out* h_plan = nullptr;  // pinned
  int* h_err = nullptr;            // pinned
  unsigned long long* d_counter = nullptr;
  int* d_work = nullptr;  // work-queue counters of the persistent kernels (kWorkSlots)
  int64_t chunk_floor = 64;
  fmt_mixed_bufs mx;
  fmt_status sticky = FMT_OK;
  char msg[256] = {0};
  // every device allocation, freed together
  void** allocs = nullptr;
  int n_allocs = 0, cap_allocs = 0;
};

// The sizes a level's kernels test their indices against.
// Whether a mixed level refits its nearly square nodes (fmt_mixed_hard) with
// Householder from the start: only when they are few enough to run in one
// wave beside the tensor-core tier (two CTAs on each of the 152 SMs), where
// that costs the level nothing and spares it the later fallbacks, which run
// one after another at its end.  Many such nodes (a forest of small problems)
// are left to the tiers, which fit most of them at far fewer FP64 flops.
constexpr int64_t kHardRouteMax = 2 * 152;
inline bool route_hard(const fmt_tree* t, int depth) {
  const int64_t h = t->lv[depth].n_hard_items;
  return t->P.precision == FMT_MIXED && h > 0 && h <= kHardRouteMax;
}

inline fmt_bounds level_bounds(const fmt_tree* t, int depth) {
  const fmt_level& L = t->lv[depth];
  fmt_bounds b;
  b.n_points = t->n;
  b.n_nodes = L.n_nodes;
  b.n_items = L.n_items;
  b.r_cap = L.r_total;
  b.n_problems = (int32_t)t->n_problems;
  b.max_m = L.max_m;
  return b;
}

// Records msg as the calling thread's last error (fmt_last_error(NULL)).
fmt_status fmt_set_error(fmt_status st, const char* msg);

// Raises the dynamic shared-memory limit of kernel `func` on the current
// device to at least `bytes` (cudaFuncAttributeMaxDynamicSharedMemorySize),
// never lowering it.  The limit belongs to the function in each context, not
// to a launch: threads that launch the same kernel with different needs (the
// serving engine's worker slots, or any caller fitting trees from several
// threads) must not lower it between another thread's setting and launch.
cudaError_t fmt_smem_at_least(const void* func, size_t bytes);

// ---------------------------------------------------------------------------
// Launchers (return cudaGetLastError() of the launch).

// build
cudaError_t launch_check_maxabs(int64_t n, const double* x, const double* y, const double* z,
                                const double* f, const fmt_problem* prob, int P, unsigned long long* d_maxbits,
                                int* d_err, cudaStream_t s);
cudaError_t launch_morton(int64_t n, const double* x, const double* y, const double* z, const fmt_problem* prob,
                          int P, int sort_shift, int sort_bits, bool key64, void* keys, uint32_t* vals,
                          cudaStream_t s);
size_t radix_sort_temp_bytes(int64_t n, bool key64);
cudaError_t launch_radix_sort(int64_t n, int bits, bool key64, void* keys, uint32_t* vals, void* keys_alt,
                              uint32_t* vals_alt, void* temp, void** keys_out, uint32_t** vals_out,
                              cudaStream_t s);
cudaError_t launch_gather(int64_t n, const uint32_t* perm, const double* x, const double* y,
                          const double* z, const double* f, const fmt_problem* prob, int P, double* xs, double* ys,
                          double* zs, double* rs, uint64_t* code, cudaStream_t s);
cudaError_t launch_plan_root(const fmt_tree* t, int64_t chunk_rows_fixed, int64_t chunk_floor,
                             fmt_plan_out* d_plan, cudaStream_t s);

// fit
int qr_rows_per_block(int m);  // the built-in rule for rows per QR block
// QR launch configuration of a level whose largest node has m columns (the
// autotuner's entry for that degree, else the built-in rule)
struct QRConfig {
  int rows, warps, chunk_factor, merge;
};
QRConfig qr_config(int m);
constexpr size_t kQRSmemMax = 227 * 1024 - 64;  // dynamic shared memory of one QR CTA
fmt_status tune_install(const fmt_tune_entry& e);  // FMT_EINVAL on a bad entry
fmt_tune_entry tune_current(int degree);
int qr_resident_ctas(int m);  // SMs x resident QR CTAs per SM
size_t qr_smem_bytes(int m, int rows);
// mode 0: every node not fitted by the mixed path; 1: only the mixed path's
// small-pivot nodes (refitted early); 2: mode 0 without those and without the
// nearly square nodes (fmt_mixed_hard); 3: only the nearly square nodes (at
// the start of a mixed level).
cudaError_t launch_tile_qr(fmt_tree* t, int depth, double* R, cudaStream_t s, int mode = 0);  // may create side streams
cudaError_t launch_combine(const fmt_tree* t, int depth, int tree_level, double* R, cudaStream_t s);
cudaError_t launch_backsolve(const fmt_tree* t, int depth, double* R, cudaStream_t s);
// r <- r - Lambda F in FP64 for the nodes of degree >= min_degree
cudaError_t launch_residual(const fmt_tree* t, int depth, cudaStream_t s, int min_degree = 0);
cudaError_t launch_child_stats(const fmt_tree* t, int depth, cudaStream_t s);

// refine / evaluate
cudaError_t launch_refine(const fmt_tree* t, int depth, int64_t chunk_rows_fixed, int64_t chunk_floor,
                          fmt_plan_out* d_plan, cudaStream_t s);
cudaError_t launch_evaluate(const fmt_tree* t, int64_t m, const int32_t* tprob, const double* xq,
                            const double* yq, const double* zq, double* out, unsigned long long* d_outside,
                            cudaStream_t s);
// mixed precision (fmt_mixed.cu)
int mixed_m_cap(int max_m);            // largest m a mixed node of the level can have
size_t mixed_acc_stride(int max_m);    // doubles of Gram accumulator per work item
// a bounded mbarrier wait that nothing satisfies (fmt_wait_probe)
cudaError_t launch_wait_probe(unsigned long long limit_ns, int* d_err, cudaStream_t s);
// the mixed path's FP64 normal-equations tier (fmt_mixed.cu): Gram, factor,
// and the sweeps' parts 0 (residual), 1 (projection), 2 (update)
cudaError_t launch_tier2_gram(const fmt_tree* t, int depth, const fmt_mixed_bufs& b, cudaStream_t s);
cudaError_t launch_tier2_factor(const fmt_tree* t, int depth, const fmt_mixed_bufs& b, cudaStream_t s);
cudaError_t launch_tier2_sweep(const fmt_tree* t, int depth, const fmt_mixed_bufs& b, int part, bool last,
                               cudaStream_t s);
cudaError_t launch_mixed_box(const fmt_tree* t, int depth, const fmt_mixed_bufs& b, cudaStream_t s);
// cache_mode: 0 generate the basis digits, 1 generate and store them (Gram), 2 load them (projection);
// without a cache buffer every launch generates
cudaError_t launch_mixed_gram(const fmt_tree* t, int depth, const fmt_mixed_bufs& b, bool projection,
                              int cache_mode, cudaStream_t s);
size_t mixed_cache_bytes(const fmt_tree* t, int depth);  // device bytes of the basis cache of a level
cudaError_t launch_mixed_factor(const fmt_tree* t, int depth, const fmt_mixed_bufs& b, cudaStream_t s);
cudaError_t launch_mixed_sresid(const fmt_tree* t, int depth, const fmt_mixed_bufs& b, cudaStream_t s);
// r <- r - Lambda F of a mixed level's nodes of degree <= FMT_MIXED_MAX_DEGREE (double-float Horner)
cudaError_t launch_mixed_final_residual(const fmt_tree* t, int depth, const fmt_mixed_bufs& b, cudaStream_t s);
cudaError_t launch_mixed_update(const fmt_tree* t, int depth, const fmt_mixed_bufs& b, bool last,
                                cudaStream_t s);
cudaError_t launch_probe_dfma(int64_t iters, int blocks, double* out, cudaStream_t s);
cudaError_t launch_check_probe(int i, int n, cudaStream_t s);  // fmt_check_probe's kernel
// Checked build: synchronise and report a failed bounds check (FMT_EINTERNAL,
// message on t, or the thread's when t is NULL); FMT_OK in the default build.
fmt_status check_end(fmt_tree* t, cudaStream_t s);
cudaError_t launch_make_hcoef(const fmt_tree* t, int depth, cudaStream_t s);
// ccoef (and ccoef_df) of a level from its hcoef and the parent level's ccoef
cudaError_t launch_make_cum(const fmt_tree* t, int depth, cudaStream_t s);
