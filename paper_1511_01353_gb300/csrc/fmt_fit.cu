// fmt_fit.cu -- fit_level kernels (Alg. 2 for all active nodes of a level).
//
// Per node, the least-squares fit of the residual over the geometric-moment
// basis is a Householder QR of the augmented matrix [Lambda(u) | r]
// (Alg. 2: DGEQRF, then F = R^{-1} Q^T f).  Q is never formed: the reflectors
// act on the last column, which ends up holding Q^T r.
//
// GB300 mapping.  The FP64 pipe is the bottleneck (about 1/60 of the FP32
// rate, and a masked lane still costs a full slot), so the kernels keep every
// FP64 instruction full-warp and avoid cross-lane reductions on the long
// loops:
//  * k_tile_qr: persistent CTAs take work items (chunks of <= C rows of one
//    node) from a queue ordered largest first; a level with several degrees
//    runs one launch per degree, on side streams.  An item's triangle R
//    (m x m, m = nmono+1) lives in global memory (L2); row blocks of 4*RPT
//    rows of [Lambda | r] are generated into shared memory and absorbed by a
//    structured Householder step per column j (the reflector touches R's row
//    j and the block's rows).  Threads form quads: a quad owns a column for
//    the whole block, each lane a quarter of the block's rows, so a column's
//    dot product needs only two shuffle-adds.  Groups of eight columns
//    belong to one warp each, and there is no barrier per step: each warp
//    schedules its own groups (the task that finalises the next pivot
//    column first) and waits only for reflectors, which the owner of each
//    pivot column publishes through a shared-memory counter (absorb_owned).
//  * k_merge / k_merge_cl / k_combine: pairwise reduction of the triangles
//    of a node (TSQR).  k_merge holds the second triangle packed in shared
//    memory (m <= 166); k_merge_cl spreads one merge over a cluster of 2-8
//    CTAs at the upper tree levels (few pairs in flight), column groups
//    owned by warps and reflectors published through shared-memory counters
//    and read over distributed shared memory; k_combine absorbs the second
//    triangle in row blocks, for any m.  The launch
//    configuration table (rows per block, warps, chunk floor, merge kernel)
//    is per degree, built in or autotuned.
//  * k_backsolve: one warp per node, column-oriented back substitution.
//  * k_residual: r <- r - Lambda F in Horner form (nmono FMAs per point).
//  * k_child_bounds / k_child_sums: octant ranges by binary search on the
//    sorted Morton codes and deterministic sums of squared residuals.
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include <cooperative_groups.h>
#include <map>
#include <mutex>
#include <utility>

#include "fmt_internal.cuh"

namespace {

constexpr int kQRThreads = 128;
int ld_for(int m);

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_maxd(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_sumi(int v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct QRArgs {
  const int64_t* item_node;
  const int64_t* item_start;
  const int64_t* item_end;
  const int32_t* item_local;
  const int32_t* node_nitems;
  const uint64_t* prefix;
  const int32_t* node_prob;
  const fmt_problem* prob;
  const double* x;
  const double* y;
  const double* z;
  const double* r;
  int depth;
  int ld_max;       // shared-memory pitch for the level's largest m
  const int64_t* item_roff;  // offset of each item's triangle in R
  double* R;
  const int32_t* sched;
  int* work;
  int n_items;
  const int32_t* flags;  // nodes with FMT_FLAG_MIXED are already fitted (mixed path)
  int only_m;            // tile QR: > 0 takes only the items of nodes with this m
  int* err;              // device error word (a bounded wait that ran out sets FMT_ERR_TIMEOUT)
  int node_mode;         // tile QR: which nodes it takes (launch_tile_qr's mode)
  const int* work_base;  // the tree's d_work (kPivSlot: the level's small-pivot count)
  const int64_t* node_start;  // the level's node point ranges (the checked build's tests;
  const int64_t* node_count;  // the count also picks the mixed path's nearly square nodes)
  fmt_bounds bd;
  int route_hard;             // route_hard(): the level sends its nearly square nodes straight to Householder
};

#ifdef FMT_CHECKED
__device__ __forceinline__ bool qr_item_ok(const QRArgs& a, int64_t item);
// Checked build: the second item of a merge pair is a valid item of the same node.
__device__ __forceinline__ bool merge_pair_ok(const QRArgs& a, int64_t item, int step) {
  return qr_item_ok(a, item + step) && a.item_node[item + step] == a.item_node[item];
}
// the node's m (its problem and degree already checked)
__device__ __forceinline__ int geo_m_of(const QRArgs& a, int64_t node) {
  const fmt_problem& pr = a.prob[a.node_prob[node]];
  return fmt_nmono_d(a.depth == 0 ? pr.q_root : pr.degree) + 1;
}

// Checked build: the item's node, problem, degree, rows (inside its node's,
// inside the points) and m x m triangle (inside the level's QR scratch).
__device__ __forceinline__ bool qr_item_ok(const QRArgs& a, int64_t item) {
  if (!fmt_in(item, a.bd.n_items)) return false;
  const int64_t node = a.item_node[item];
  if (!fmt_in(node, a.bd.n_nodes) || !fmt_in(a.node_prob[node], a.bd.n_problems)) return false;
  const fmt_problem& pr = a.prob[a.node_prob[node]];
  const int q = a.depth == 0 ? pr.q_root : pr.degree;
  if (pr.degree > FMT_MAX_DEGREE || q < 0 || q > pr.degree) return false;
  const int64_t m = fmt_nmono_d(q) + 1, ro = a.item_roff[item];
  if (m > a.bd.max_m || ro < 0 || ro + m * m > a.bd.r_cap) return false;
  const int64_t s = a.node_start[node], e = s + a.node_count[node];
  const int64_t rs = a.item_start[item], re = a.item_end[item];
  return 0 <= s && s <= rs && rs <= re && re <= e && e <= a.bd.n_points;
}
#endif

// A node the mixed path's tensor-core tier left for a small Cholesky pivot:
// eligible for that tier (degree <= FMT_MIXED_MAX_DEGREE, not a clamped root),
// FMT_FLAG_MIXED_PIVOT and no FMT_FLAG_MIXED_SLOW (the FP64 tier, which
// runs later, sets the pivot flag only on nodes that were not eligible or
// did not converge).  These are known right after the factor kernel.
// Both launches read the level's count of such nodes (kPivSlot, written by
// the factor kernel) and take the early path only when it is at most
// kEarlyRefitMax, so they agree on which nodes the early launch takes.
__device__ __forceinline__ bool early_refit(const QRArgs& a, int64_t node, int32_t f) {
  const fmt_problem& pr = a.prob[a.node_prob[node]];
  const bool eligible = pr.degree <= FMT_MIXED_MAX_DEGREE && !(a.depth == 0 && pr.q_root < pr.degree);
  return eligible && (f & (FMT_FLAG_MIXED | FMT_FLAG_MIXED_SLOW | FMT_FLAG_MIXED_PIVOT)) == FMT_FLAG_MIXED_PIVOT &&
         a.work_base[kPivSlot] <= kEarlyRefitMax;
}

// A node the mixed path sends straight to Householder (on a level that
// routes them): of a degree its tiers cover, not a clamped root, nearly
// square (fmt_mixed_hard).
__device__ __forceinline__ bool hard_node(const QRArgs& a, int64_t node) {
  const fmt_problem& pr = a.prob[a.node_prob[node]];
  return a.route_hard && pr.degree <= FMT_MIXED_FP64_MAX_DEGREE && !(a.depth == 0 && pr.q_root < pr.degree) &&
         fmt_mixed_hard(pr.degree, a.node_count[node]);
}

__device__ __forceinline__ bool node_done(const QRArgs& a, int64_t node) {
  const int32_t f = a.flags[node];
  if (f & FMT_FLAG_MIXED) return true;
  if (a.node_mode == 3) return !hard_node(a, node);
  if (a.node_mode == 1) return !early_refit(a, node, f);
  if (a.node_mode == 2) return early_refit(a, node, f) || hard_node(a, node);
  return false;
}

// degree, column count and frame of a node of the level
struct NodeGeom {
  int q, m, ldB;
  double c0, s0, c1, s1, c2, s2;
};
__device__ __forceinline__ NodeGeom node_geom(const QRArgs& a, int64_t node) {
  NodeGeom g;
  const fmt_problem& pr = a.prob[a.node_prob[node]];
  g.q = a.depth == 0 ? pr.q_root : pr.degree;
  g.m = fmt_nmono_d(g.q) + 1;
  g.ldB = fmt_ld_for(g.m);
  const uint64_t pf = fmt_morton_part(a.prefix[node], a.depth);
  fmt_frame(pr.lo[0], pr.side, pr.inv_side, a.depth, fmt_compact3(pf), g.c0, g.s0);
  fmt_frame(pr.lo[1], pr.side, pr.inv_side, a.depth, fmt_compact3(pf >> 1), g.c1, g.s1);
  fmt_frame(pr.lo[2], pr.side, pr.inv_side, a.depth, fmt_compact3(pf >> 2), g.c2, g.s2);
  return g;
}

// Structured Householder absorb of a row block B (NB x m in shared memory,
// leading dimension ldB) into the upper triangle R (m x m, row-major, global).
// For each column j >= j_begin: alpha = R_jj, x = B[:, j],
// beta = -sign(alpha) sqrt(alpha^2 + |x|^2) (sign(0) = +), u = [alpha - beta; x]
// and H = I - gamma u u^T, gamma = 1 / (h (h + |alpha|)), h = |beta|: the
// update of a column [rv; b] is d = gamma (amb rv + x.b), rv -= d amb,
// b -= d x with amb = alpha - beta.  Where h h nears underflow (the rounding
// residue left in a block's columns beyond its rank, whose squares go
// subnormal at degree >= 12) gamma would overflow, so there the column is
// scaled in place to v = x / amb and (gamma, amb) = (tau, 1) with LAPACK's
// tau = 1 + |alpha| / h in [1, 2]: the same formula, nothing over- or
// underflows.  A column with |x| = 0 is left alone (gamma = 0).
//
// Schedule per step j (one barrier per step):
//  * row j of R sits in shared memory (Rs[j&1]); row j+1 was prefetched into
//    registers during step j-1 and is stashed into Rs[(j+1)&1] here, while
//    row j+2 is fetched from global memory for the next step;
//  * quads update the columns k > j (round r covers 32 columns); updated R_jk
//    are written through to global memory;
//  * warp 0, right after its first round (which updates column j+1), computes
//    the reflector of step j+1 (look-ahead), so no step waits on a serial
//    norm / sqrt / divide phase of its own.
// The scalars of a reflector from alpha and s = |x|^2 (every lane of the
// warp computes them: lane-0-only FP64 code costs the same issue slots).
// Returns the factor to scale x by (0: none).
__device__ __forceinline__ double refl_scalars(double alpha, double s, double& gamma, double& amb, double& beta) {
  const double h = sqrt(fma(alpha, alpha, s));
  beta = alpha >= 0.0 ? -h : h;
  const double hpa = h + fabs(alpha);  // |alpha - beta|
  if (h > 0x1p-400) {
    gamma = 1.0 / (h * hpa);
    amb = alpha - beta;
    return 0.0;
  }
  gamma = hpa / h;  // tau
  amb = 1.0;
  return alpha >= 0.0 ? 1.0 / hpa : -1.0 / hpa;
}

// One warp: gamma and amb of column j into sc, beta into R_jj (shared row and
// global R).
__device__ __forceinline__ void reflector(double* __restrict__ B, int ldB, int NB, int j, double* Rrow,
                                          double* __restrict__ Rg, int m, double* sc) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < NB; i += 32) {
    const double xv = B[i * ldB + j];
    s = fma(xv, xv, s);
  }
  s = warp_sum(s);  // the same value in every lane (butterfly)
  const double alpha = Rrow[j];
  __syncwarp();  // every lane has read R_jj before it is overwritten
  if (s == 0.0) {
    if (lane == 0) {
      sc[0] = 0.0;
      sc[1] = 0.0;
    }
    return;
  }
  double gamma, amb, beta;
  const double scale = refl_scalars(alpha, s, gamma, amb, beta);
  if (scale != 0.0)
    for (int i = lane; i < NB; i += 32) B[i * ldB + j] *= scale;
  if (lane == 0) {
    sc[0] = gamma;
    sc[1] = amb;
    Rrow[j] = beta;
    Rg[(size_t)j * m + j] = beta;
  }
}

// tri_row0 >= 0 marks a block whose row i is zero left of column tri_row0+i
// (rows of another triangle): at step j only rows i <= j - tri_row0 can be
// nonzero, so whole groups of four rows are skipped (warp-uniform bound).
template <int RPT, int NW>
__device__ __forceinline__ void absorb_block(double* __restrict__ B, int ldB, int j_begin, int m,
                                             double* __restrict__ R, double* __restrict__ Rs, double* sc,
                                             int tri_row0) {
  constexpr int NB = 4 * RPT;
  constexpr int NT = 32 * NW;
  constexpr int kPF = (680 + NT - 1) / NT;  // enough prefetch registers for degree 14
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, rg = tid & 3;
  if (j_begin >= m) return;
  // prologue: row j_begin into shared memory, its reflector, prefetch of the next row
  for (int k = j_begin + tid; k < m; k += NT) Rs[(j_begin & 1) * ldB + k] = R[(size_t)j_begin * m + k];
  __syncthreads();
  if (warp == 0) reflector(B, ldB, NB, j_begin, Rs + (j_begin & 1) * ldB, R, m, sc + (j_begin & 1) * 2);
  static_assert((NW & (NW - 1)) == 0, "warp count must be a power of two");
  // The look-ahead warp of step j is lw(j) = (j + blockIdx.x) mod NW.  Row j+1
  // is prefetched and stashed with the thread index rotated so that lane 0 of
  // lw(j) holds its first element R_{j+1,j+1}: the look-ahead then reads it
  // after a __syncwarp, without a block barrier.
  auto rot = [&](int jj) { return (tid - 32 * ((jj + (int)blockIdx.x) & (NW - 1))) & (NT - 1); };
  double pf[kPF];
  {
    const int rt = rot(j_begin);
#pragma unroll
    for (int e = 0; e < kPF; ++e) {
      const int k = j_begin + 1 + rt + NT * e;
      pf[e] = (k < m) ? R[(size_t)(j_begin + 1) * m + k] : 0.0;
    }
  }
  __syncthreads();
  for (int j = j_begin; j < m; ++j) {
    const int cur = j & 1, nxt = cur ^ 1;
    double* Rc = Rs + cur * ldB;
    double* Rn = Rs + nxt * ldB;
    {
      const int rs = rot(j);  // row j+1 was fetched with this mapping
#pragma unroll
      for (int e = 0; e < kPF; ++e) {
        const int k = j + 1 + rs + NT * e;
        if (k < m) Rn[k] = pf[e];
      }
      const int rp = rot(j + 1);  // row j+2 is stashed at step j+1
#pragma unroll
      for (int e = 0; e < kPF; ++e) {
        const int k = j + 2 + rp + NT * e;
        pf[e] = (k < m) ? R[(size_t)(j + 2) * m + k] : 0.0;
      }
    }
    // groups of four rows that can hold nonzeros at this step (warp uniform)
    const int tmax = tri_row0 < 0 ? RPT : min(RPT, max(0, (j - tri_row0) / 4 + 1));
    const double gamma = sc[cur * 2], amb = sc[cur * 2 + 1];
    const bool upd = gamma != 0.0;
    double xr[RPT];
    if (upd) {
#pragma unroll
      for (int t = 0; t < RPT; ++t) xr[t] = (t < tmax) ? B[(rg + 4 * t) * ldB + j] : 0.0;
    }
    // The warp roles rotate with the step (and differ between CTAs): the warp
    // with slot 0 takes columns j+1..j+8 of each round and the look-ahead, so
    // the extra work does not always land on the same SM sub-partition.
    const int slot = (warp - j - (int)blockIdx.x) & (NW - 1);
    int k0 = j + 1 + 8 * slot;  // columns j+1+8*slot .. j+8+8*slot of each round
    bool lookahead = (slot == 0) && (j + 1 < m);
    for (;;) {
      if (upd && k0 < m) {
        const int k = k0 + (lane >> 2);
        const bool act = k < m;
        const int kk = act ? k : j;
        double acc;
        if (NW <= 4) {
          // pipe-bound (several rounds per step): one chain, since the DFMA
          // latency is below the FP64 issue interval and the join add is saved
          acc = 0.0;
#pragma unroll
          for (int t = 0; t < RPT; ++t)
            if (t < tmax) acc = fma(xr[t], B[(rg + 4 * t) * ldB + kk], acc);
        } else {
          // latency-bound (about one round per step): two chains
          double a0 = 0.0, a1 = 0.0;
#pragma unroll
          for (int t = 0; t < RPT; t += 2) {
            if (t < tmax) a0 = fma(xr[t], B[(rg + 4 * t) * ldB + kk], a0);
            if (t + 1 < tmax) a1 = fma(xr[t + 1], B[(rg + 4 * t + 4) * ldB + kk], a1);
          }
          acc = a0 + a1;
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        if (act) {
          const double rv = Rc[k];
          const double d = gamma * fma(amb, rv, acc);
#pragma unroll
          for (int t = 0; t < RPT; ++t) {
            if (t < tmax) {
              double* bp = B + (rg + 4 * t) * ldB + k;
              *bp = fma(-d, xr[t], *bp);
            }
          }
          if (rg == 0) R[(size_t)j * m + k] = fma(-d, amb, rv);
        }
        k0 += 8 * NW;
      }
      if (lookahead) {  // column j+1 is final for this step: reflector of step j+1
        __syncwarp();
        reflector(B, ldB, NB, j + 1, Rn, R, m, sc + nxt * 2);
        lookahead = false;
        continue;
      }
      if (!upd || k0 >= m) break;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- owned absorb
// The tile QR's absorb of a row block B (NB x m, shared) into R (m x m,
// global), with no barrier per Householder step.  Column k belongs to quad
// k & 7 of warp own(k >> 3) for the whole block (groups of eight columns
// dealt round robin over the warps, rotated from block to block), so the
// updates of a column by reflectors 0, 1, 2, ... are done in order by one
// quad and a warp waits only for the reflector of the step it is at.  The
// owner of column j+1 applies reflector j to its group first, then forms
// reflector j+1 and publishes it (scalars in scv[2(j+1)], scv[2(j+1)+1];
// R_{j+1,j+1} = beta; column j+1 of B is final) by raising *pub to j+2.
// A warp at step j: waits for *pub > j (bounded: the wait sets
// FMT_ERR_TIMEOUT and *abort on expiry, and every warp then leaves the
// block), then updates every column k > j it owns:
// d = gamma (amb R_jk + x . b_k), R_jk -= d amb, b_k -= d x.
// Compared with one barrier per step, a warp with no column left at a step
// goes on to the next step as soon as its reflector is out, so a step's last
// partial round of 8 NW columns costs no idle lanes in the other warps.
constexpr long long kOwnSpinMax = 1ll << 26;  // polls of one wait (about a second)

__device__ __forceinline__ void own_reflector(double* __restrict__ B, int ldB, int NB, int j,
                                              double* __restrict__ Rg, int m, double* scv) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < NB; i += 32) {
    const double xv = B[i * ldB + j];
    s = fma(xv, xv, s);
  }
  s = warp_sum(s);
  const double alpha = Rg[(size_t)j * m + j];
  __syncwarp();  // every lane has read R_jj before it is overwritten
  if (s == 0.0) {
    if (lane == 0) {
      scv[2 * j] = 0.0;
      scv[2 * j + 1] = 0.0;
    }
    return;
  }
  double gamma, amb, beta;
  const double scale = refl_scalars(alpha, s, gamma, amb, beta);
  if (scale != 0.0)
    for (int i = lane; i < NB; i += 32) B[i * ldB + j] *= scale;
  if (lane == 0) {
    scv[2 * j] = gamma;
    scv[2 * j + 1] = amb;
    Rg[(size_t)j * m + j] = beta;
  }
}

// Raises *pub to v once every lane's writes are visible to the block.
__device__ __forceinline__ void own_publish(volatile int* pub, int v) {
  __threadfence_block();
  __syncwarp();
  if ((threadIdx.x & 31) == 0) *pub = v;
}

// Waits (lane 0, bounded) until *pub >= v and returns the value seen (in
// every lane; the reflectors below it are visible to the warp), or -1 if
// the block is aborting.
__device__ __forceinline__ int own_wait(volatile int* pub, int v, volatile int* abort_flag, int* err) {
  int seen = -1;
  if ((threadIdx.x & 31) == 0) {
    long long spins = 0;
    for (;;) {
      const int p = *pub;
      if (p >= v) {
        seen = p;
        break;
      }
      if (*abort_flag) break;
      if (++spins > kOwnSpinMax) {
        atomicOr(err, FMT_ERR_TIMEOUT);
        *abort_flag = 1;
        break;
      }
    }
    __threadfence_block();
  }
  seen = __shfl_sync(0xffffffffu, seen, 0);
  __syncwarp();  // orders the other lanes' reads after lane 0's wait
  return seen;
}

// Owner table of the column groups for m columns: longest first, each group
// (work: the sum of its column indices, one update per earlier step) to the
// warp with the least work so far (the busiest warp ends 1% above the mean
// at m = 166 with 4 warps, 10% with 8; round robin 7% and 28%).  Also the
// groups of every table warp in ascending order (list / start / count).
// One thread.
constexpr int kMaxGroups = (FMT_MAX_DEGREE + 1) * (FMT_MAX_DEGREE + 2) * (FMT_MAX_DEGREE + 3) / 6 / 8 + 1;
struct OwnTab {
  unsigned char own[kMaxGroups];   // table warp of each group
  unsigned char list[kMaxGroups];  // groups by table warp, ascending
  unsigned char start[8], count[8];
};
template <int NW>
__device__ void own_table(int m, OwnTab& T) {
  const int ng = (m + 7) >> 3;
  int load[NW];
  for (int w = 0; w < NW; ++w) load[w] = 0;
  for (int g = ng - 1; g >= 0; --g) {  // the cost grows with g: descending g is longest first
    const int k1 = 8 * g + 8 < m ? 8 * g + 8 : m;
    const int cost = (8 * g + k1 - 1) * (k1 - 8 * g) / 2;
    int best = 0;
    for (int w = 1; w < NW; ++w)
      if (load[w] < load[best]) best = w;
    T.own[g] = (unsigned char)best;
    load[best] += cost;
  }
  int o = 0;
  for (int w = 0; w < NW; ++w) {
    T.start[w] = (unsigned char)o;
    for (int g = 0; g < ng; ++g)
      if (T.own[g] == w) T.list[o++] = (unsigned char)g;
    T.count[w] = (unsigned char)(o - T.start[w]);
  }
}

// Lane 0 reads the published count; broadcast to the warp.  No fence: a
// warp fences (own_acquire) before it first uses a reflector it has seen.
__device__ __forceinline__ int own_peek(volatile int* pub) {
  int v = 0;
  if ((threadIdx.x & 31) == 0) v = *pub;
  return __shfl_sync(0xffffffffu, v, 0);
}
__device__ __forceinline__ void own_acquire() {
  if ((threadIdx.x & 31) == 0) __threadfence_block();
  __syncwarp();
}

// Every warp runs its own schedule over the groups it owns: the task
// "apply reflector ver[g] to group g" is ready once that reflector is
// published.  The task that makes the next reflector final (the group of
// column P, P reflectors published, at version P-1) goes first, so the
// owner of column j+1 publishes reflector j+1 as soon as reflector j is
// out, whatever else it still has to do; otherwise the ready task of the
// lowest version.  A warp with nothing ready waits for the next reflector.
// Lane i of a warp keeps the version of the warp's i-th group in a
// register; one warp-wide minimum picks the task.
template <int RPT, int NW>
__device__ __forceinline__ bool absorb_owned(double* __restrict__ B, int ldB, int m, double* __restrict__ R,
                                             double* __restrict__ scv, volatile int* pub, volatile int* abort_flag,
                                             int rotw, const OwnTab& T, int* err) {
  constexpr int NB = 4 * RPT;
  static_assert((NW & (NW - 1)) == 0, "warp count must be a power of two");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, rg = lane & 3, qi = lane >> 2;
  const int tw = (warp - rotw) & (NW - 1);  // this warp's row of the table
  const int gn = T.count[tw];               // at most 32 groups per warp (m <= 681, 4+ warps)
  const int mg = lane < gn ? T.list[T.start[tw] + lane] : -1;  // the group this lane tracks
  const int mk = mg >= 0 ? (8 * mg + 7 < m - 1 ? 8 * mg + 7 : m - 1) : 0;  // reflectors it needs
  int mv = 0;                                                             // reflectors applied to it
  int P = 0, Pacq = 0;  // reflectors seen published / acquired (visible) by this warp
  if (((T.own[0] + rotw) & (NW - 1)) == warp) {
    own_reflector(B, ldB, NB, 0, R, m, scv);
    own_publish(pub, 1);
    P = Pacq = 1;
  }
  for (;;) {
    const bool live = mg >= 0 && mv < mk;
    if (!__any_sync(0xffffffffu, live)) break;
    // key: -1 for the critical task, else the version of a ready task
    int key = 0x7fffffff;
    if (live && mv < P) key = (mv == P - 1 && mg == (P >> 3)) ? -1 : mv;
    const int kmin = __reduce_min_sync(0xffffffffu, key);
    if (kmin == 0x7fffffff) {  // nothing ready: the next reflector
      const int seen = own_wait(pub, P + 1, abort_flag, err);
      if (seen < 0) return false;
      P = Pacq = seen;
      continue;
    }
    const int src = __ffs(__ballot_sync(0xffffffffu, key == kmin)) - 1;
    const int sel = __shfl_sync(0xffffffffu, mg, src);
    const int j = __shfl_sync(0xffffffffu, mv, src);
    if (j >= Pacq) {
      own_acquire();
      Pacq = P;
    }
    const double gamma = scv[2 * j], amb = scv[2 * j + 1];
    if (gamma != 0.0) {
      double xr[RPT];
#pragma unroll
      for (int t = 0; t < RPT; ++t) xr[t] = B[(rg + 4 * t) * ldB + j];
      const int k = 8 * sel + qi;
      const bool act = k > j && k < m;
      const int kk = act ? k : j;  // inactive quads read a valid column
      const double rv = act ? R[(size_t)j * m + k] : 0.0;
      double acc = 0.0;
#pragma unroll
      for (int t = 0; t < RPT; ++t) acc = fma(xr[t], B[(rg + 4 * t) * ldB + kk], acc);
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      if (act) {
        const double d = gamma * fma(amb, rv, acc);
#pragma unroll
        for (int t = 0; t < RPT; ++t) {
          double* bp = B + (rg + 4 * t) * ldB + k;
          *bp = fma(-d, xr[t], *bp);
        }
        if (rg == 0) R[(size_t)j * m + k] = fma(-d, amb, rv);
      }
    }
    if (lane == src) mv = j + 1;
    if (((j + 1) >> 3) == sel) {  // column j+1 is final: reflector j+1
      __syncwarp();
      own_reflector(B, ldB, NB, j + 1, R, m, scv);
      own_publish(pub, j + 2);
      if (P < j + 2) P = Pacq = j + 2;
    } else {
      const int v = own_peek(pub);
      if (v > P) P = v;
    }
  }
  return true;
}

// Persistent CTAs take work items from a queue in the order of `sched`
// (largest items first), so the longest chunks start early.  NW warps per
// CTA (the autotuner picks 4 or 8).  Shared memory: the row block (NB x
// ld_max), then the reflector scalars of every step (2 ld_max >= 2 m).
template <int RPT, int NW>
__global__ void __launch_bounds__(32 * NW, NW >= 8 ? 2 : 1) k_tile_qr(QRArgs a) {
  extern __shared__ double smem[];
  constexpr int NB = 4 * RPT, NT = 32 * NW;
  static_assert(NB <= NT, "one thread generates each row of a block");
  double* Bs = smem;
  double* scv = smem + NB * a.ld_max;
  __shared__ int s_item;
  __shared__ int s_pub, s_abort, s_own_m;
  __shared__ OwnTab s_own;
  if (threadIdx.x == 0) {
    s_abort = 0;
    s_own_m = -1;
  }
  int nblk = 0;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(a.work, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= a.n_items) break;
    const int item = a.sched[it];
    if (!FMT_CHECK(qr_item_ok(a, item), CK_QR_ITEM)) continue;
    const int64_t node = a.item_node[item];
    if (node_done(a, node)) continue;
    const int64_t rs = a.item_start[item], re = a.item_end[item];
    const NodeGeom g = node_geom(a, node);
    if (a.only_m > 0 && g.m != a.only_m) continue;  // another degree's launch takes it
    if (!FMT_CHECK(g.ldB <= a.ld_max, CK_QR_ITEM)) continue;
    const int m = g.m, q = g.q, ldB = g.ldB;
    double* R = a.R + a.item_roff[item];
    if (threadIdx.x == 0 && s_own_m != m) {  // the items of a launch share m except a clamped root
      own_table<NW>(m, s_own);
      s_own_m = m;
    }
    for (int e = threadIdx.x; e < m * m; e += NT) {
      const int j = e / m, k = e - j * m;
      if (k >= j) R[e] = 0.0;
    }
    __syncthreads();
    for (int64_t b0 = rs; b0 < re; b0 += NB) {
      const int nb = (int)((re - b0) < NB ? (re - b0) : NB);
      if (threadIdx.x < NB) {
        double* row = Bs + threadIdx.x * ldB;
        if ((int)threadIdx.x < nb) {
          const int64_t i = b0 + threadIdx.x;
          const double u = fmt_local(a.x[i], g.c0, g.s0), v = fmt_local(a.y[i], g.c1, g.s1),
                       w = fmt_local(a.z[i], g.c2, g.s2);
          double pu[FMT_MAX_DEGREE + 1], pv[FMT_MAX_DEGREE + 1], pw[FMT_MAX_DEGREE + 1];
          double tu = 1.0, tv = 1.0, tw = 1.0;
          for (int l = 0; l <= q; ++l) {
            const double f = c_invfact[l];
            pu[l] = tu * f;
            pv[l] = tv * f;
            pw[l] = tw * f;
            tu *= u;
            tv *= v;
            tw *= w;
          }
          int k = 0;
          for (int l = 0; l <= q; ++l)
            for (int mm = 0; mm <= q - l; ++mm) {
              const double plm = pu[l] * pv[mm];
              for (int n = 0; n <= q - l - mm; ++n) row[k++] = plm * pw[n];
            }
          row[k] = a.r[i];
        } else {
          for (int k = 0; k < m; ++k) row[k] = 0.0;
        }
      }
      if (threadIdx.x == 0) s_pub = 0;
      __syncthreads();
      absorb_owned<RPT, NW>(Bs, ldB, m, R, scv, &s_pub, &s_abort, (nblk + (int)blockIdx.x) & (NW - 1), s_own,
                            a.err);
      ++nblk;
      __syncthreads();  // the block is absorbed (or abandoned): the next one may overwrite it
      if (s_abort) return;
    }
  }
}

// Pairwise merge of two triangles of one node (a TSQR tree level): the second
// triangle is absorbed into the first in blocks of NB rows.  Few pairs are
// active at the top of the tree, so this kernel runs 16 warps per CTA.
constexpr int kCombineWarps = 16;
template <int RPT>
__global__ void __launch_bounds__(32 * kCombineWarps) k_combine(QRArgs a, int level) {
  extern __shared__ double smem[];
  constexpr int NB = 4 * RPT;
  double* Bs = smem;
  double* Rs = smem + NB * a.ld_max;
  double* sc = Rs + 2 * a.ld_max;
  const int item = blockIdx.x;
  if (!FMT_CHECK(qr_item_ok(a, item), CK_MERGE_ITEM)) return;
  const int s = a.item_local[item];
  const int64_t node = a.item_node[item];
  const int cnt = a.node_nitems[node];
  const int step = 1 << level;
  if ((s & (2 * step - 1)) != 0 || s + step >= cnt || node_done(a, node)) return;
  if (!FMT_CHECK(merge_pair_ok(a, item, step), CK_MERGE_ITEM)) return;
  const NodeGeom g = node_geom(a, node);
  const int m = g.m;
  double* Ra = a.R + a.item_roff[item];
  const double* Rb = a.R + a.item_roff[item + step];
  for (int r0 = 0; r0 < m; r0 += NB) {
    for (int e = threadIdx.x; e < NB * m; e += 32 * kCombineWarps) {
      const int i = e / m, k = e - i * m;
      const int row = r0 + i;
      Bs[i * g.ldB + k] = (row < m && k >= row) ? Rb[(size_t)row * m + k] : 0.0;
    }
    __syncthreads();
    absorb_block<RPT, kCombineWarps>(Bs, g.ldB, r0, m, Ra, Rs, sc, r0);
  }
}

// Pairwise merge with the whole second triangle in shared memory, stored
// column by column (column k of the upper triangle, rows 0..k, starts at
// k(k+1)/2), so that the rows of a column are contiguous: one pass of m
// Householder steps.  Step j reflects row j of R_a with rows 0..j of R_b
// (rows below j are still zero in column j); columns k > j are updated by
// quads whose four lanes split the rows 0..j.  R_a's rows are streamed
// through shared memory with a one-step prefetch.  The m steps form a chain
// (reflector j+1 needs column j+1 after step j), so one warp per step
// finalises column j+1 with all its lanes and forms reflector j+1 while the
// other warps update the columns past it.  Used when the packed triangle
// fits in shared memory (m <= 166 with two CTAs per SM); the merge is
// latency-bound, so it runs 16 warps.
constexpr int kMergeWarps = 16;
constexpr int kMergeThreads = 32 * kMergeWarps;

__global__ void __launch_bounds__(kMergeThreads) k_merge(QRArgs a, int level) {
  extern __shared__ double smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, rg = tid & 3;
  const int item = blockIdx.x;
  if (!FMT_CHECK(qr_item_ok(a, item), CK_MERGE_ITEM)) return;
  const int sidx = a.item_local[item];
  const int cnt = a.node_nitems[a.item_node[item]];
  const int step = 1 << level;
  if ((sidx & (2 * step - 1)) != 0 || sidx + step >= cnt || node_done(a, a.item_node[item])) return;
  if (!FMT_CHECK(merge_pair_ok(a, item, step), CK_MERGE_ITEM)) return;
  const NodeGeom g = node_geom(a, a.item_node[item]);
  const int m = g.m;
  double* Ra = a.R + a.item_roff[item];
  const double* Rb = a.R + a.item_roff[item + step];
  const int ldR = g.ldB;
  double* Bp = smem;                                   // R_b, packed by columns
  double* Rs = Bp + ((m * (m + 1) / 2 + 1) & ~1);      // two rows of R_a
  double* sc = Rs + 2 * ldR;                           // reflector scalars of two steps
  for (int k = warp; k < m; k += kMergeWarps) {
    const int cb = k * (k + 1) / 2;
    for (int i = lane; i <= k; i += 32) Bp[cb + i] = Rb[(size_t)i * m + k];
  }
  for (int k = tid; k < m; k += kMergeThreads) Rs[k] = Ra[k];  // row 0 of R_a
  __syncthreads();

  // Reflector j from column j of R_b (rows 0..j), sq = its squared norm
  // (the same value in every lane) and R_a[j][j]; one warp, as reflector().
  auto reflect = [&](int j, double* Rrow, double* scj, double sq) {
    double* col = Bp + j * (j + 1) / 2;
    const double alpha = Rrow[j];
    __syncwarp();
    if (sq == 0.0) {
      if (lane == 0) {
        scj[0] = 0.0;
        scj[1] = 0.0;
      }
      return;
    }
    double gamma, amb, beta;
    const double scale = refl_scalars(alpha, sq, gamma, amb, beta);
    if (scale != 0.0)
      for (int i = lane; i <= j; i += 32) col[i] *= scale;
    if (lane == 0) {
      scj[0] = gamma;
      scj[1] = amb;
      Rrow[j] = beta;
      Ra[(size_t)j * m + j] = beta;
    }
  };
  auto rot = [&](int jj) { return (tid - 32 * ((jj + (int)blockIdx.x) & (kMergeWarps - 1))) & (kMergeThreads - 1); };
  constexpr int kPF = (680 + kMergeThreads - 1) / kMergeThreads;
  if (warp == 0) reflect(0, Rs, sc, Bp[0] * Bp[0]);
  double pf[kPF];
  {
    const int rt = rot(0);
#pragma unroll
    for (int e = 0; e < kPF; ++e) {
      const int k = 1 + rt + kMergeThreads * e;
      pf[e] = (k < m) ? Ra[(size_t)1 * m + k] : 0.0;
    }
  }
  __syncthreads();
  // Step j: the warp of slot 0 finalises column j+1 alone (all 32 lanes on its
  // rows 0..j, then its norm) and forms reflector j+1: the chain of dependent
  // steps runs through that warp only, a few full-warp instructions per
  // step.  The other warps update columns j+2 .. m-1 in quads, eight columns
  // per warp and round.
  for (int j = 0; j < m; ++j) {
    const int cur = j & 1, nxt = cur ^ 1;
    double* Rc = Rs + cur * ldR;
    double* Rn = Rs + nxt * ldR;
    {
      const int rs = rot(j);
#pragma unroll
      for (int e = 0; e < kPF; ++e) {
        const int k = j + 1 + rs + kMergeThreads * e;
        if (k < m) Rn[k] = pf[e];  // the slot-0 warp's lane 0 writes Rn[j + 1]
      }
      const int rp = rot(j + 1);
#pragma unroll
      for (int e = 0; e < kPF; ++e) {
        const int k = j + 2 + rp + kMergeThreads * e;
        pf[e] = (k < m) ? Ra[(size_t)(j + 2) * m + k] : 0.0;
      }
    }
    const double gamma = sc[cur * 2], amb = sc[cur * 2 + 1];
    const bool upd = gamma != 0.0;
    const double* xj = Bp + j * (j + 1) / 2;  // column j, rows 0..j
    const int slot = (warp - j - (int)blockIdx.x) & (kMergeWarps - 1);
    if (slot == 0) {
      if (j + 1 < m) {
        double* cn = Bp + (j + 1) * (j + 2) / 2;  // column j+1
        double sq = 0.0;
        if (upd) {
          double acc = 0.0;
          for (int i = lane; i <= j; i += 32) acc = fma(xj[i], cn[i], acc);
          acc = warp_sum(acc);
          const double rv = Rc[j + 1];
          const double d = gamma * fma(amb, rv, acc);
          for (int i = lane; i <= j; i += 32) {
            const double nv = fma(-d, xj[i], cn[i]);
            cn[i] = nv;
            sq = fma(nv, nv, sq);
          }
          if (lane == 0) Ra[(size_t)j * m + j + 1] = fma(-d, amb, rv);
        } else {
          for (int i = lane; i <= j; i += 32) sq = fma(cn[i], cn[i], sq);
        }
        if (lane == 0) sq = fma(cn[j + 1], cn[j + 1], sq);  // row j+1: no step has touched it
        sq = warp_sum(sq);
        __syncwarp();  // lane 0's Rn[j + 1] is visible to the warp
        reflect(j + 1, Rn, sc + nxt * 2, sq);
      }
    } else if (upd) {
      for (int k0 = j + 2 + 8 * (slot - 1); k0 < m; k0 += 8 * (kMergeWarps - 1)) {
        const int k = k0 + (lane >> 2);
        const bool act = k < m;
        double* ck = Bp + (act ? k * (k + 1) / 2 : j * (j + 1) / 2);  // column k (column j when idle)
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int i = rg;
        for (; i + 12 <= j; i += 16) {
          a0 = fma(xj[i], ck[i], a0);
          a1 = fma(xj[i + 4], ck[i + 4], a1);
          a2 = fma(xj[i + 8], ck[i + 8], a2);
          a3 = fma(xj[i + 12], ck[i + 12], a3);
        }
        for (; i <= j; i += 4) a0 = fma(xj[i], ck[i], a0);
        double acc = (a0 + a1) + (a2 + a3);
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        if (act) {
          const double rv = Rc[k];
          const double d = gamma * fma(amb, rv, acc);
          int i2 = rg;
          for (; i2 + 12 <= j; i2 += 16) {
            const double b0 = fma(-d, xj[i2], ck[i2]);
            const double b1 = fma(-d, xj[i2 + 4], ck[i2 + 4]);
            const double b2 = fma(-d, xj[i2 + 8], ck[i2 + 8]);
            const double b3 = fma(-d, xj[i2 + 12], ck[i2 + 12]);
            ck[i2] = b0;
            ck[i2 + 4] = b1;
            ck[i2 + 8] = b2;
            ck[i2 + 12] = b3;
          }
          for (; i2 <= j; i2 += 4) ck[i2] = fma(-d, xj[i2], ck[i2]);
          if (rg == 0) Ra[(size_t)j * m + k] = fma(-d, amb, rv);
        }
      }
    }
    __syncthreads();
  }
}

size_t merge_smem_bytes(int m) {
  return ((size_t)((m * (m + 1) / 2 + 1) & ~1) + 2 * (size_t)ld_for(m) + 4) * sizeof(double);
}

// ---------------------------------------------------------------- cluster merge
// The merge of two triangles [R_a; R_b] (a TSQR tree level) by a cluster of
// C CTAs: the top levels of a node's merge tree hold few pairs, and one merge
// on one SM is a chain of m dependent Householder steps, so there the steps
// are spread over C SMs.  Columns come in groups of W = 32 / LW (LW lanes per
// column); each group belongs to one warp of one CTA, which keeps the
// group's columns of R_b and of R_a (rows 0 .. W g + W - 1, both upper
// triangular; step j touches rows 0..j of R_b and row j of R_a) in its
// shared memory for the whole merge and writes R_a back at the end.  Step
// j's reflector is formed from column j by the warp that owns it as soon as
// reflector j-1 has reached that column: its scalars stay in the owner
// CTA's shared memory and a counter in every CTA is raised by a release
// reduction.  A warp applies reflector j to its groups once the counter of
// its own CTA passes j (acquire load), reading the reflector's scalars and
// vector from the owner CTA's shared memory (distributed shared memory).  Each warp schedules its
// groups as absorb_owned does: the task that finalises the next pivot
// column first, else the oldest ready one.  In that task all 32 lanes
// update the pivot column and form its reflector, which is published before
// the group's other columns are updated, so the chain of m dependent steps
// costs a few full-warp instructions per step.  Waits are bounded (kOwnSpinMax
// polls; FMT_ERR_TIMEOUT).  C = 1 is the same kernel on one SM.
namespace cg = cooperative_groups;
constexpr int kMCWarps = 8;
constexpr int kMCMaxM = 287;  // degree <= 10
constexpr int kMCMaxGroups = kMCMaxM;

struct MCLayout {
  unsigned char own_cta[kMCMaxGroups], own_warp[kMCMaxGroups];
  int off[kMCMaxGroups];                 // offset (doubles) of the group's blocks in its CTA's block area
  unsigned short list[kMCMaxGroups];     // groups by owner (cta-major), ascending
  unsigned short start[8 * kMCWarps], count[8 * kMCWarps];
  int cta_doubles[8];                    // block area of each CTA
};

// Longest-first over the C * kMCWarps owners (owner o: CTA o % C, warp o / C,
// so consecutive owners sit on different SMs); work of group g ~ (W g + W)^2.
// A group's blocks: R_b part then R_a part, (W g + W) rows of W doubles each.
__host__ __device__ inline bool mc_layout(int m, int C, int W, MCLayout& L) {
  const int ng = (m + W - 1) / W, no = C * kMCWarps;
  if (ng > kMCMaxGroups) return false;
  long long load[8 * kMCWarps];
  for (int o = 0; o < no; ++o) load[o] = 0;
  unsigned short own_o[kMCMaxGroups];
  for (int g = ng - 1; g >= 0; --g) {
    int best = 0;
    for (int o = 1; o < no; ++o)
      if (load[o] < load[best]) best = o;
    own_o[g] = (unsigned short)best;
    load[best] += (long long)(W * g + W) * (W * g + W);
  }
  for (int c = 0; c < 8; ++c) L.cta_doubles[c] = 0;
  for (int g = 0; g < ng; ++g) {
    const int o = own_o[g], c = o % C;
    L.own_cta[g] = (unsigned char)c;
    L.own_warp[g] = (unsigned char)(o / C);
    L.off[g] = L.cta_doubles[c];
    L.cta_doubles[c] += 2 * (W * g + W) * W;
  }
  int n = 0;
  for (int c = 0; c < C; ++c)
    for (int w = 0; w < kMCWarps; ++w) {
      L.start[c * kMCWarps + w] = (unsigned short)n;
      for (int g = 0; g < ng; ++g)
        if (L.own_cta[g] == c && L.own_warp[g] == w) L.list[n++] = (unsigned short)g;
      L.count[c * kMCWarps + w] = (unsigned short)(n - L.start[c * kMCWarps + w]);
      if (L.count[c * kMCWarps + w] > 32) return false;  // one lane tracks each group of a warp
    }
  return true;
}

__host__ __device__ inline int mc_scv_doubles(int m) { return (2 * m + 1) & ~1; }

__device__ __forceinline__ uint32_t mc_smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Raise the counter at shared address `laddr` of CTA `rank` to at least v,
// after this thread's earlier writes (and those ordered before it) are
// visible to the cluster (C > 1) or the CTA.
template <int C>
__device__ __forceinline__ void mc_raise(uint32_t laddr, int rank, int v) {
  if (C > 1) {
    uint32_t raddr;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(raddr) : "r"(laddr), "r"(rank));
    asm volatile("red.release.cluster.shared::cluster.max.s32 [%0], %1;" ::"r"(raddr), "r"(v) : "memory");
  } else {
    asm volatile("red.release.cta.shared::cta.max.s32 [%0], %1;" ::"r"(laddr), "r"(v) : "memory");
  }
}
template <int C>
__device__ __forceinline__ int mc_read(uint32_t laddr) {
  int v;
  if (C > 1)
    asm volatile("ld.acquire.cluster.shared::cta.b32 %0, [%1];" : "=r"(v) : "r"(laddr) : "memory");
  else
    asm volatile("ld.acquire.cta.shared::cta.b32 %0, [%1];" : "=r"(v) : "r"(laddr) : "memory");
  return v;
}

template <int C, int LW>
__global__ void __launch_bounds__(32 * kMCWarps) k_merge_cl(QRArgs a, int level) {
  constexpr int W = 32 / LW;  // columns per group (one per LW lanes)
  extern __shared__ double smem[];
  __shared__ MCLayout L;
  __shared__ int s_pub, s_abort;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, rg = lane % LW, qi = lane / LW;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = C > 1 ? (int)cl.block_rank() : 0;
  const int item = (int)(blockIdx.x / C);
  // every CTA of a cluster takes the same decisions
  if (!FMT_CHECK(qr_item_ok(a, item), CK_MERGE_ITEM)) return;
  const int sidx = a.item_local[item];
  const int64_t node = a.item_node[item];
  const int cnt = a.node_nitems[node];
  const int step = 1 << level;
  if ((sidx & (2 * step - 1)) != 0 || sidx + step >= cnt || node_done(a, node)) return;
  if (!FMT_CHECK(merge_pair_ok(a, item, step) && geo_m_of(a, node) <= kMCMaxM, CK_MERGE_ITEM)) return;
  const NodeGeom geo = node_geom(a, node);
  const int m = geo.m;
  double* Ra = a.R + a.item_roff[item];
  const double* Rb = a.R + a.item_roff[item + step];
  double* scv = smem;                      // gamma_j, amb_j of every step
  double* vbuf = smem + mc_scv_doubles(m); // per warp: a copy of another CTA's pivot column (m doubles)
  double* blk = vbuf + kMCWarps * m;       // this CTA's group blocks
  if (tid == 0) {
    mc_layout(m, C, W, L);
    s_pub = 0;
    s_abort = 0;
  }
  __syncthreads();
  const int ng = (m + W - 1) / W;
  for (int g = 0; g < ng; ++g) {
    if (L.own_cta[g] != rank) continue;
    const int rows = W * g + W;
    double* b = blk + L.off[g];
    for (int e = tid; e < rows * W; e += 32 * kMCWarps) {
      const int i = e / W, k = W * g + (e % W);
      const bool in = k < m && i <= k;
      b[e] = in ? Rb[(size_t)i * m + k] : 0.0;
      b[rows * W + e] = in ? Ra[(size_t)i * m + k] : 0.0;
    }
  }
  __syncthreads();
  if (C > 1) cl.sync();  // every CTA's blocks and counter are set before any remote access
  const uint32_t pub_addr = mc_smem_u32(&s_pub);
  volatile int* vab = &s_abort;

  auto cta_ptr = [&](double* p, int c) -> double* { return C > 1 ? cl.map_shared_rank(p, c) : p; };
  auto kmax = [&](int g) { return W * g + W - 1 < m - 1 ? W * g + W - 1 : m - 1; };
  // Reflector j from column j of its group (this warp) and R_a[j][j]; the
  // scalars to every CTA, then the counters.
  // s = |rows 0..j of R_b's column j|^2, the same value in every lane.
  auto reflect_publish = [&](int j, double s) {
    const int gj = j / W, cj = j % W, rows = W * gj + W;
    double* col = blk + L.off[gj] + cj;  // R_b row i at col[W i], R_a row i at col[W (rows + i)]
    double* ajj = col + W * (rows + j);
    const double alpha = *ajj;
    __syncwarp();
    double gamma = 0.0, amb = 0.0, beta;
    if (s != 0.0) {
      const double scale = refl_scalars(alpha, s, gamma, amb, beta);
      if (scale != 0.0)
        for (int i = lane; i <= j; i += 32) col[W * i] *= scale;
      if (lane == 0) *ajj = beta;
    }
    if (lane == 0) {  // the scalars stay with the owner; other CTAs read them remotely
      scv[2 * j] = gamma;
      scv[2 * j + 1] = amb;
    }
    __syncwarp();
    if (lane < C) mc_raise<C>(pub_addr, lane, j + 1);
  };

  const int ow = rank * kMCWarps + warp;
  const int gn = L.count[ow];
  const int mg = lane < gn ? L.list[L.start[ow] + lane] : -1;
  const int mk = mg >= 0 ? kmax(mg) : 0;
  int mv = 0;
  int P = 0;
  int vcopy = -1;  // the remote pivot column this warp's buffer holds
  if (L.own_cta[0] == rank && L.own_warp[0] == warp) {
    const double b00 = blk[L.off[0]];
    reflect_publish(0, b00 * b00);
    P = 1;
  }
  for (;;) {
    const bool live = mg >= 0 && mv < mk;
    if (!__any_sync(0xffffffffu, live)) break;
    int key = 0x7fffffff;
    // the critical task, else the oldest ready one (ties: the group needed soonest)
    if (live && mv < P) key = (mv == P - 1 && mg == P / W) ? -1 : (mv << 10) | mg;
    const int kmin = __reduce_min_sync(0xffffffffu, key);
    if (kmin == 0x7fffffff) {  // nothing ready: wait for the next reflector
      int seen = -1;
      if (lane == 0) {
        long long spins = 0;
        for (;;) {
          const int pv = mc_read<C>(pub_addr);
          if (pv > P) {
            seen = pv;
            break;
          }
          if (*vab) break;
          if (++spins > kOwnSpinMax) {
            atomicOr(a.err, FMT_ERR_TIMEOUT);
            *vab = 1;
            break;
          }
        }
      }
      seen = __shfl_sync(0xffffffffu, seen, 0);
      __syncwarp();
      if (seen < 0) break;  // aborting: leave through the cluster barrier
      P = seen;
      continue;
    }
    const int srcl = __ffs(__ballot_sync(0xffffffffu, key == kmin)) - 1;
    const int sel = __shfl_sync(0xffffffffu, mg, srcl);
    const int j = __shfl_sync(0xffffffffu, mv, srcl);
    const int gj = j / W, oj = L.own_cta[gj];
    const double* sj = oj == rank ? scv : cta_ptr(scv, oj);
    const double gamma = sj[2 * j], amb = sj[2 * j + 1];
    const int rows = W * sel + W;
    const bool crit = (j + 1) / W == sel;  // column j+1 is in this group: the task finalises it
    const int cq = (j + 1) % W;
    const double* vj = blk + L.off[gj] + (j % W);  // v_i at vj[vs i]
    int vs = W;
    if (gamma != 0.0 && oj != rank) {
      // another CTA's column: one pipelined pass of remote loads into this
      // warp's buffer (kept while the warp stays on the same reflector)
      double* lv = vbuf + warp * m;
      if (vcopy != j) {
        const double* rv_ = cta_ptr(blk + L.off[gj], oj) + (j % W);
        for (int i = lane; i <= j; i += 32) lv[i] = rv_[W * i];
        __syncwarp();
        vcopy = j;
      }
      vj = lv;
      vs = 1;
    }
    if (crit) {
      // column j+1 by all 32 lanes (its rows 0..j and its norm), then
      // reflector j+1: the chain of dependent steps passes through here
      double* cc = blk + L.off[sel] + cq;  // R_b row i at cc[W i]
      double sq = 0.0;
      if (gamma != 0.0) {
        double* ac = cc + W * (rows + j);  // R_a[j][j+1]
        const double rvc = *ac;
        double acc = 0.0;
        for (int i = lane; i <= j; i += 32) acc = fma(vj[vs * i], cc[W * i], acc);
        acc = warp_sum(acc);
        const double d = gamma * fma(amb, rvc, acc);
        for (int i = lane; i <= j; i += 32) {
          const double nv = fma(-d, vj[vs * i], cc[W * i]);
          cc[W * i] = nv;
          sq = fma(nv, nv, sq);
        }
        __syncwarp();  // every lane has read R_a[j][j+1]
        if (lane == 0) *ac = fma(-d, amb, rvc);
      } else {
        // no reflection at step j: column j+1's rows 0..j are unchanged
        for (int i = lane; i <= j; i += 32) sq = fma(cc[W * i], cc[W * i], sq);
      }
      const double s = warp_sum(sq);
      const double bjj = cc[W * (j + 1)];  // row j+1 of column j+1 (no step has touched it)
      __syncwarp();
      reflect_publish(j + 1, fma(bjj, bjj, s));
      if (P < j + 2) P = j + 2;
    }
    // the group's columns past j (past j+1 when column j+1 was done above), LW lanes each
    if (gamma != 0.0 && !(crit && cq == W - 1)) {
      double* ck = blk + L.off[sel] + qi;  // R_b column W sel + qi: row i at ck[W i]
      double* ak = ck + W * (rows + j);    // R_a[j][W sel + qi]
      const int k = W * sel + qi;
      const bool act = k > (crit ? j + 1 : j) && k < m;
      const double rv = *ak;
      double a0 = 0.0, a1 = 0.0;
      int i = rg;
      for (; i + LW <= j; i += 2 * LW) {
        a0 = fma(vj[vs * i], ck[W * i], a0);
        a1 = fma(vj[vs * (i + LW)], ck[W * (i + LW)], a1);
      }
      if (i <= j) a0 = fma(vj[vs * i], ck[W * i], a0);
      double acc = a0 + a1;
#pragma unroll
      for (int o = 1; o < LW; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (act) {
        const double d = gamma * fma(amb, rv, acc);
        for (int i2 = rg; i2 <= j; i2 += LW) ck[W * i2] = fma(-d, vj[vs * i2], ck[W * i2]);
        if (rg == 0) *ak = fma(-d, amb, rv);
      }
    }
    if (lane == srcl) mv = j + 1;
    if (!crit) {
      int v = 0;
      if (lane == 0) v = mc_read<C>(pub_addr);
      v = __shfl_sync(0xffffffffu, v, 0);
      __syncwarp();
      if (v > P) P = v;
    }
  }
  __syncthreads();
  // R_a back to global memory: the owned columns, rows 0..k
  for (int g = 0; g < ng; ++g) {
    if (L.own_cta[g] != rank) continue;
    const int rows = W * g + W;
    const double* b = blk + L.off[g] + rows * W;
    for (int e = tid; e < rows * W; e += 32 * kMCWarps) {
      const int i = e / W, k = W * g + (e % W);
      if (k < m && i <= k) Ra[(size_t)i * m + k] = b[e];
    }
  }
  if (C > 1) cl.sync();  // no CTA leaves while another may still read its blocks or raise its counter
}

// Dynamic shared memory of the cluster merge with C CTAs (the largest CTA's
// share), or 0 if the layout does not exist or a share exceeds 200 KB.
size_t merge_cl_smem_bytes(int m, int C, int W) {
  if (m > kMCMaxM) return 0;
  MCLayout L;
  if (!mc_layout(m, C, W, L)) return 0;
  int mx = 0;
  for (int c = 0; c < C; ++c) mx = L.cta_doubles[c] > mx ? L.cta_doubles[c] : mx;
  const size_t b = ((size_t)mc_scv_doubles(m) + (size_t)kMCWarps * m + (size_t)mx) * sizeof(double);
  return b <= 200 * 1024 ? b : 0;
}

template <int C, int LW>
cudaError_t merge_cl_launch(const QRArgs& a, int64_t n_items, size_t smem, int level, cudaStream_t s) {
  cudaError_t e = fmt_smem_at_least((const void*)k_merge_cl<C, LW>, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n_items * C));
  cfg.blockDim = dim3(32 * kMCWarps);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, k_merge_cl<C, LW>, a, level);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// ---------------------------------------------------------------- back solve
struct BSArgs {
  int64_t n_nodes;
  const int64_t* node_item0;
  const int64_t* item_roff;
  double* R;
  int depth;
  const int32_t* node_prob;
  const fmt_problem* prob;
  int stride;  // coefficients per node (nmono of the largest degree)
  int ws;      // back-solve workspace per warp (doubles)
  double* coef;
  double* hcoef;
  int32_t* flags;
  int32_t* deg_used;
  int64_t n_items;
  fmt_bounds bd;
};

__device__ __forceinline__ int tri2(int k) { return (k + 1) * (k + 2) / 2; }

// (l, m, n) of the idx-th monomial of degree <= p in Alg. 2 order
__device__ void mono_lmn(int p, int idx, int& l, int& m, int& n) {
  l = 0;
  while (idx >= tri2(p - l)) {
    idx -= tri2(p - l);
    ++l;
  }
  m = 0;
  while (idx >= p - l - m + 1) {
    idx -= p - l - m + 1;
    ++m;
  }
  n = idx;
}
__device__ int mono_index(int p, int l, int m, int n) {
  int idx = 0;
  for (int a = 0; a < l; ++a) idx += tri2(p - a);
  for (int b = 0; b < m; ++b) idx += p - l - b + 1;
  return idx + n;
}

// Back substitution of one node by one warp: F = R^{-1} (Q^T r) on the final
// triangle [R | Q^T r] (m x m, row-major), with the rank rule (columns with
// |R_jj| <= 64 L eps max|R_kk| dropped and the rest re-triangularised).
// Writes F and F / (l! m! n!) in the degree-p layout (zeros for monomials of
// degree > q and for dropped columns).  ws: 3L + (L+1)/2 + 1 doubles.
// Returns the number of dropped columns.
__device__ int backsolve_warp(double* __restrict__ R, int m, int q, int p, int nmono_p, double* ws,
                              double* __restrict__ cf, double* __restrict__ hc) {
  const int lane = threadIdx.x & 31;
  const int L = m - 1;
  double* y = ws;
  double* inv = y + L;
  double* F = inv + L;
  int* keep = (int*)(F + L);

  double rmax = 0.0;
  for (int j = lane; j < L; j += 32) rmax = fmax(rmax, fabs(R[(size_t)j * m + j]));
  rmax = warp_maxd(rmax);
  const double thresh = 64.0 * (double)L * DBL_EPSILON * rmax;
  int ndrop = 0;
  for (int j = lane; j < L; j += 32) ndrop += fabs(R[(size_t)j * m + j]) <= thresh ? 1 : 0;
  ndrop = warp_sumi(ndrop);
  int Lk = L;
  if (ndrop > 0) {
    // Rank rule: drop dependent columns, re-triangularise [R_kept | Q^T r].
    int c = 0;
    for (int j0 = 0; j0 < L; j0 += 32) {
      const int j = j0 + lane;
      const bool kp = j < L && fabs(R[(size_t)j * m + j]) > thresh;
      const unsigned b = __ballot_sync(0xffffffffu, kp);
      if (kp) keep[c + __popc(b & ((1u << lane) - 1u))] = j;
      c += __popc(b);
    }
    Lk = c;
    __syncwarp();
    for (int i = lane; i < m; i += 32) {
      for (int cc = 0; cc < Lk; ++cc) {
        const int src = keep[cc];
        R[(size_t)i * m + cc] = (i <= src) ? R[(size_t)i * m + src] : 0.0;
      }
      R[(size_t)i * m + Lk] = R[(size_t)i * m + L];
    }
    __syncwarp();
    for (int cc = 0; cc <= Lk && cc < m; ++cc) {
      const int rmx = (cc < Lk) ? keep[cc] : L;
      const double alpha = R[(size_t)cc * m + cc];
      double s = 0.0;
      for (int i = cc + 1 + lane; i <= rmx; i += 32) {
        const double t = R[(size_t)i * m + cc];
        s = fma(t, t, s);
      }
      s = warp_sum(s);
      if (s == 0.0) continue;
      // reflector in the normalised form of reflector(): v over the column
      const double h = sqrt(fma(alpha, alpha, s));
      const double beta = alpha >= 0.0 ? -h : h;
      const double tau = (h + fabs(alpha)) / h;
      const double inv = 1.0 / (alpha - beta);
      for (int i = cc + 1 + lane; i <= rmx; i += 32) R[(size_t)i * m + cc] *= inv;
      __syncwarp();
      for (int k = cc + 1 + lane; k <= Lk; k += 32) {
        double w = R[(size_t)cc * m + k];
        for (int i = cc + 1; i <= rmx; ++i) w = fma(R[(size_t)i * m + cc], R[(size_t)i * m + k], w);
        const double d = tau * w;
        R[(size_t)cc * m + k] -= d;
        for (int i = cc + 1; i <= rmx; ++i) R[(size_t)i * m + k] = fma(-d, R[(size_t)i * m + cc], R[(size_t)i * m + k]);
      }
      __syncwarp();
      if (lane == 0) R[(size_t)cc * m + cc] = beta;
      for (int i = cc + 1 + lane; i <= rmx; i += 32) R[(size_t)i * m + cc] = 0.0;
      __syncwarp();
    }
  }
  for (int j = lane; j < Lk; j += 32) {
    const double dg = R[(size_t)j * m + j];
    y[j] = R[(size_t)j * m + Lk];
    inv[j] = fabs(dg) <= thresh ? 0.0 : 1.0 / dg;
  }
  __syncwarp();
  for (int j = Lk - 1; j >= 0; --j) {
    const double Fj = y[j] * inv[j];
    if (lane == 0) F[j] = Fj;
    for (int k = lane; k < j; k += 32) y[k] = fma(-R[(size_t)k * m + j], Fj, y[k]);
    __syncwarp();
  }
  if (q != p || ndrop > 0) {
    for (int k = lane; k < nmono_p; k += 32) {
      cf[k] = 0.0;
      hc[k] = 0.0;
    }
    __syncwarp();
  }
  for (int c = lane; c < Lk; c += 32) {
    const int jq = ndrop > 0 ? keep[c] : c;
    int l, mm, n;
    mono_lmn(q, jq, l, mm, n);
    const int jp = (q == p) ? jq : mono_index(p, l, mm, n);
    cf[jp] = F[c];
    hc[jp] = F[c] * (c_invfact[l] * c_invfact[mm] * c_invfact[n]);
  }
  __syncwarp();
  return ndrop;
}

__host__ __device__ inline int backsolve_ws_doubles(int L) { return 3 * L + (L + 1) / 2 + 1; }

#ifdef FMT_CHECKED
// Checked build: the node's problem and degree, its first item's triangle
// inside the QR scratch, its coefficients inside the node's slot and its m
// within the workspace the launch sized.
__device__ __forceinline__ bool backsolve_node_ok(const BSArgs& a, int64_t node) {
  if (!fmt_in(a.node_prob[node], a.bd.n_problems)) return false;
  const fmt_problem& pr = a.prob[a.node_prob[node]];
  const int q = a.depth == 0 ? pr.q_root : pr.degree;
  if (pr.degree > FMT_MAX_DEGREE || q < 0 || q > pr.degree || fmt_nmono_d(pr.degree) > a.stride) return false;
  const int64_t m = fmt_nmono_d(q) + 1, i0 = a.node_item0[node];
  if (m > a.bd.max_m || !fmt_in(i0, a.bd.n_items)) return false;
  const int64_t ro = a.item_roff[i0];
  return ro >= 0 && ro + m * m <= a.bd.r_cap;
}
#endif

__global__ void __launch_bounds__(128) k_backsolve(BSArgs a) {
  extern __shared__ double sm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t node = (int64_t)blockIdx.x * 4 + wib;
  if (node >= a.n_nodes) return;
  if (a.flags[node] & FMT_FLAG_MIXED) return;  // fitted by the mixed path
  if (!FMT_CHECK(backsolve_node_ok(a, node), CK_BACKSOLVE_NODE)) return;  // one warp per node
  const fmt_problem& pr = a.prob[a.node_prob[node]];
  const int p = pr.degree;
  const int q = a.depth == 0 ? pr.q_root : p;
  const int m = fmt_nmono_d(q) + 1;
  const int nmono_p = fmt_nmono_d(p);
  double* ws = sm + (size_t)wib * a.ws;
  double* R = a.R + a.item_roff[a.node_item0[node]];
  double* cf = a.coef + (size_t)node * a.stride;
  double* hc = a.hcoef + (size_t)node * a.stride;
  const int ndrop = backsolve_warp(R, m, q, p, nmono_p, ws, cf, hc);
  for (int k = nmono_p + lane; k < a.stride; k += 32) {  // lower-degree problems in a forest
    cf[k] = 0.0;
    hc[k] = 0.0;
  }
  if (lane == 0) {
    a.deg_used[node] = q;
    if (ndrop > 0) a.flags[node] |= FMT_FLAG_RANK;
  }
}

// ---------------------------------------------------------------- residual
struct ResArgs {
  const int64_t* item_node;
  const int64_t* item_start;
  const int64_t* item_end;
  const uint64_t* prefix;
  const int32_t* node_prob;
  const fmt_problem* prob;
  const double* x;
  const double* y;
  const double* z;
  double* r;
  const double* hcoef;
  int depth, stride;
  const int64_t* node_start;  // checked build
  const int64_t* node_count;
  fmt_bounds bd;
  int min_degree;  // nodes of lower degree are skipped (their residual is computed elsewhere)
};

#ifdef FMT_CHECKED
// Checked build: the item's node, problem and degree, and its rows inside
// its node's inside the points.
__device__ __forceinline__ bool residual_item_ok(const ResArgs& a, int64_t item) {
  const int64_t node = a.item_node[item];
  if (!fmt_in(node, a.bd.n_nodes) || !fmt_in(a.node_prob[node], a.bd.n_problems)) return false;
  const int p = a.prob[a.node_prob[node]].degree;
  if (p < 0 || p > FMT_MAX_DEGREE || fmt_nmono_d(p) > a.stride) return false;
  const int64_t s = a.node_start[node], e = s + a.node_count[node];
  const int64_t rs = a.item_start[item], re = a.item_end[item];
  return 0 <= s && s <= rs && rs <= re && re <= e && e <= a.bd.n_points;
}
#endif

__global__ void __launch_bounds__(256) k_residual(ResArgs a) {
  const int item = blockIdx.x;
  if (!FMT_CHECK(residual_item_ok(a, item), CK_RESIDUAL_ITEM)) return;
  const int64_t node = a.item_node[item];
  const int64_t rs = a.item_start[item], re = a.item_end[item];
  const fmt_problem& pr = a.prob[a.node_prob[node]];
  const uint64_t pf = fmt_morton_part(a.prefix[node], a.depth);
  double c0, s0, c1, s1, c2, s2;
  fmt_frame(pr.lo[0], pr.side, pr.inv_side, a.depth, fmt_compact3(pf), c0, s0);
  fmt_frame(pr.lo[1], pr.side, pr.inv_side, a.depth, fmt_compact3(pf >> 1), c1, s1);
  fmt_frame(pr.lo[2], pr.side, pr.inv_side, a.depth, fmt_compact3(pf >> 2), c2, s2);
  const int p = pr.degree, nm = fmt_nmono_d(p);
  if (p < a.min_degree) return;
  const double* G = a.hcoef + (size_t)node * a.stride;
  for (int64_t i = rs + threadIdx.x; i < re; i += blockDim.x) {
    const double u = fmt_local(a.x[i], c0, s0), v = fmt_local(a.y[i], c1, s1), w = fmt_local(a.z[i], c2, s2);
    a.r[i] -= fmt_horner(G, p, nm, u, v, w);
  }
}

// ---------------------------------------------------------------- child stats
struct ChildArgs {
  int64_t n_nodes;
  const uint64_t* prefix;
  const int64_t* start;
  const int64_t* count;
  const uint64_t* code;
  const double* r;
  int64_t* bounds;
  double* child_S;
  int64_t* child_n;
  int shift;  // 3*(21-depth-1); < 0 when the node has no child level
  int depth;
  fmt_bounds bd;
};

__global__ void __launch_bounds__(256) k_child_bounds(ChildArgs a) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= a.n_nodes * 9) return;
  const int64_t node = gid / 9;
  const int o = (int)(gid - node * 9);
  const int64_t s = a.start[node], e = s + a.count[node];
  if (!FMT_CHECK(0 <= s && s <= e && e <= a.bd.n_points, CK_CHILD_NODE)) return;
  int64_t b;
  if (a.shift < 0) {
    b = s;  // no octants below the deepest code level
  } else if (o == 0) {
    b = s;
  } else if (o == 8) {
    b = e;
  } else {
    const uint64_t target = fmt_morton_part(a.prefix[node], a.depth) * 8ull + (uint64_t)o;
    int64_t lo = s, hi = e;
    while (lo < hi) {
      const int64_t mid = lo + ((hi - lo) >> 1);
      if ((a.code[mid] >> a.shift) < target) lo = mid + 1;
      else hi = mid;
    }
    b = lo;
  }
  a.bounds[node * 9 + o] = b;
}

__global__ void __launch_bounds__(128) k_child_sums(ChildArgs a) {
  __shared__ double red[4];
  const int64_t node = blockIdx.x >> 3;
  const int o = blockIdx.x & 7;
  const int64_t b0 = a.bounds[node * 9 + o], b1 = a.bounds[node * 9 + o + 1];
  if (!FMT_CHECK(0 <= b0 && b0 <= b1 && b1 <= a.bd.n_points, CK_CHILD_NODE)) return;  // uniform over the CTA
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int64_t i = b0 + threadIdx.x;
  for (; i + 3 * 128 < b1; i += 4 * 128) {
    const double t0 = a.r[i], t1 = a.r[i + 128], t2 = a.r[i + 256], t3 = a.r[i + 384];
    s0 = fma(t0, t0, s0);
    s1 = fma(t1, t1, s1);
    s2 = fma(t2, t2, s2);
    s3 = fma(t3, t3, s3);
  }
  for (; i < b1; i += 128) {
    const double t = a.r[i];
    s0 = fma(t, t, s0);
  }
  double s = (s0 + s1) + (s2 + s3);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    a.child_S[node * 8 + o] = (red[0] + red[1]) + (red[2] + red[3]);
    a.child_n[node * 8 + o] = b1 - b0;
  }
}

// The merges of a configuration with 128-row blocks absorb in 64-row blocks
// (16 warps of k_combine would not hold 32 rows per lane in registers); its
// shared memory is the tile QR's, which is larger.
template <int RPT>
constexpr int combine_rpt() { return RPT > 16 ? 16 : RPT; }

template <int RPT, int NW>
cudaError_t set_smem_attr(size_t smem) {
  cudaError_t e = fmt_smem_at_least((const void*)k_tile_qr<RPT, NW>, smem);
  if (e != cudaSuccess) return e;
  return fmt_smem_at_least((const void*)k_combine<combine_rpt<RPT>()>, smem);
}

int ld_for(int m) { return fmt_ld_for(m); }

QRArgs make_qr_args(const fmt_tree* t, int depth, double* R) {
  const fmt_level& L = t->lv[depth];
  QRArgs a;
  a.item_node = L.item_node;
  a.item_start = L.item_start;
  a.item_end = L.item_end;
  a.item_local = L.item_local;
  a.node_nitems = L.node_nitems;
  a.prefix = L.prefix;
  a.node_prob = L.prob;
  a.prob = t->d_prob;
  a.x = t->x;
  a.y = t->y;
  a.z = t->z;
  a.r = t->r;
  a.depth = depth;
  a.ld_max = ld_for(L.max_m);
  a.item_roff = L.item_roff;
  a.R = R;
  a.sched = L.sched;
  a.work = t->d_work;
  a.n_items = (int)L.n_items;
  a.flags = L.flags;
  a.only_m = 0;
  a.err = t->d_err;
  a.node_mode = 0;
  a.work_base = t->d_work;
  a.node_start = L.start;
  a.node_count = L.count;
  a.bd = level_bounds(t, depth);
  a.route_hard = route_hard(t, depth) ? 1 : 0;
  return a;
}

}  // namespace

int qr_rows_per_block(int m) {
  const size_t ld = (size_t)ld_for(m);
  if (66 * ld * sizeof(double) + 32 <= 110 * 1024) return 64;
  if (34 * ld * sizeof(double) + 32 <= 200 * 1024) return 32;
  return 16;
}

size_t qr_smem_bytes(int m, int rows) { return ((size_t)(rows + 2) * ld_for(m) + 4) * sizeof(double); }

// ------------------------------------------------------------ launch table
// One QR launch configuration per degree: the built-in rule, or an entry
// from the autotuner / fmt_tune_set.
namespace {
std::mutex g_tune_mu;
fmt_tune_entry g_tune[FMT_MAX_DEGREE + 1];  // zero: source 0 (built-in rule)

int degree_of_m(int m) {
  for (int p = 0; p <= FMT_MAX_DEGREE; ++p)
    if (fmt_nmono_d(p) + 1 == m) return p;
  return -1;
}

fmt_tune_entry builtin_entry(int p) {
  fmt_tune_entry e{};
  e.degree = p;
  e.rows = qr_rows_per_block(fmt_nmono_d(p) + 1);
  // 8 warps from degree 8 on: two warps per sub-partition hide more of the
  // FP64 latency of the owned-column schedule (p = 8: 300 against 305 ms of
  // tile QR per scale step; the one-degree tuner picks 8 at p = 10 to 12)
  e.warps = fmt_nmono_d(p) + 1 >= 160 ? 8 : 4;
  e.chunk_factor = 4;
  e.merge = 0;
  e.source = 0;
  return e;
}

bool entry_ok(const fmt_tune_entry& e) {
  if (e.degree < 0 || e.degree > FMT_MAX_DEGREE) return false;
  if (e.source == 0) return true;
  if (e.rows != 16 && e.rows != 32 && e.rows != 48 && e.rows != 64 && e.rows != 128) return false;
  if (e.warps != 4 && e.warps != 8) return false;
  if (e.chunk_factor != 1 && e.chunk_factor != 2 && e.chunk_factor != 4 && e.chunk_factor != 8 &&
      e.chunk_factor != 16)
    return false;
  if (e.merge != 0 && e.merge != 1) return false;
  return qr_smem_bytes(fmt_nmono_d(e.degree) + 1, e.rows) <= kQRSmemMax;
}
}  // namespace

QRConfig qr_config(int m) {
  const int p = degree_of_m(m);
  fmt_tune_entry e;
  if (p < 0) {
    e = builtin_entry(0);
    e.rows = qr_rows_per_block(m);
  } else {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    e = g_tune[p].source != 0 ? g_tune[p] : builtin_entry(p);
  }
  return QRConfig{e.rows, e.warps, e.chunk_factor, e.merge};
}

fmt_status tune_install(const fmt_tune_entry& in) {
  if (!entry_ok(in)) return FMT_EINVAL;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[in.degree] = in;
  if (in.source == 0) g_tune[in.degree] = fmt_tune_entry{};
  return FMT_OK;
}

fmt_tune_entry tune_current(int p) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return g_tune[p].source != 0 ? g_tune[p] : builtin_entry(p);
}

namespace {
template <int RPT, int NW>
int resident_for(size_t smem) {
  int per_sm = 0;
  if (set_smem_attr<RPT, NW>(smem) != cudaSuccess) return 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_qr<RPT, NW>, 32 * NW, smem) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return per_sm > 0 ? per_sm : 1;
}

template <int RPT, int NW>
cudaError_t tile_launch(const QRArgs& a, unsigned grid, size_t smem, cudaStream_t s) {
  cudaError_t e = set_smem_attr<RPT, NW>(smem);
  if (e != cudaSuccess) return e;
  k_tile_qr<RPT, NW><<<grid, 32 * NW, smem, s>>>(a);
  return cudaGetLastError();
}

template <int RPT, int NW>
cudaError_t combine_launch(const QRArgs& a, unsigned grid, size_t smem, cudaStream_t s, int level) {
  cudaError_t e = set_smem_attr<RPT, NW>(smem);
  if (e != cudaSuccess) return e;
  k_combine<combine_rpt<RPT>()><<<grid, 32 * kCombineWarps, smem, s>>>(a, level);
  return cudaGetLastError();
}

// the kernels of one (rows, warps) configuration
struct QROps {
  int (*resident)(size_t);
  cudaError_t (*tile)(const QRArgs&, unsigned, size_t, cudaStream_t);
  cudaError_t (*combine)(const QRArgs&, unsigned, size_t, cudaStream_t, int);
};
template <int RPT, int NW>
QROps ops_for() {
  return QROps{&resident_for<RPT, NW>, &tile_launch<RPT, NW>, &combine_launch<RPT, NW>};
}
QROps qr_ops(const QRConfig& c) {
  if (c.warps == 8)
    return c.rows == 128  ? ops_for<32, 8>()
           : c.rows == 64 ? ops_for<16, 8>()
           : c.rows == 48 ? ops_for<12, 8>()
           : c.rows == 32 ? ops_for<8, 8>()
                          : ops_for<4, 8>();
  return c.rows == 128  ? ops_for<32, 4>()
         : c.rows == 64 ? ops_for<16, 4>()
         : c.rows == 48 ? ops_for<12, 4>()
         : c.rows == 32 ? ops_for<8, 4>()
                        : ops_for<4, 4>();
}
}  // namespace

int qr_resident_ctas(int m) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (nsm <= 0) nsm = 1;
  const QRConfig c = qr_config(m);
  return nsm * qr_ops(c).resident(qr_smem_bytes(m, c.rows));
}

// One launch per degree present in the level, each with its degree's
// configuration, shared-memory pitch and work-queue counter, so a forest
// level mixing degrees 4..10 does not run every item with the largest
// degree's blocks.  The launches go to side streams forked from s, largest
// degree first: as one launch's persistent CTAs run out of items the next
// one's take their SMs, so the launches share one tail instead of one each.
// A level of one degree is one launch on s.
cudaError_t launch_tile_qr(fmt_tree* t, int depth, double* R, cudaStream_t s, int mode) {
  const fmt_level& L = t->lv[depth];
  const int64_t n_items = L.n_items;
  if (n_items <= 0) return cudaSuccess;
  const uint64_t mask = (uint64_t)L.deg_mask;
  const bool several = (mask & (mask - 1)) != 0;
  // the side-stream launches (modes 1 and 3, one after the other) have their own counters
  int* work0 = t->d_work + 1 + (mode == 1 || mode == 3 ? FMT_MAX_DEGREE + 1 : 0);
  auto launch_one = [&](int mq, cudaStream_t st, int* work) -> cudaError_t {
    QRArgs a = make_qr_args(t, depth, R);
    a.node_mode = mode;
    a.only_m = several ? mq : 0;
    a.ld_max = ld_for(mq);
    a.work = work;
    QRConfig c = qr_config(mq);
    // the early refits are a few small nodes beside other work: latency-bound
    // single CTAs, where 8 warps hide more of the FP64 latency than 4
    if (mode == 1 || mode == 3) c.warps = 8;
    const size_t smem = qr_smem_bytes(mq, c.rows);
    int64_t grid = qr_resident_ctas(mq);
    if (grid > n_items) grid = n_items;
    if (mode == 3 && grid > L.n_hard_items) grid = L.n_hard_items;  // only those items have work
    cudaError_t e = cudaMemsetAsync(work, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    return qr_ops(c).tile(a, (unsigned)grid, smem, st);
  };
  if (!several) return launch_one(L.max_m, s, work0);
  cudaError_t e;
  if (!t->fork_ev && (e = cudaEventCreateWithFlags(&t->fork_ev, cudaEventDisableTiming)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(t->fork_ev, s)) != cudaSuccess) return e;
  for (int q = FMT_MAX_DEGREE; q >= 0; --q) {
    if (!(mask & (1ull << q))) continue;
    if (!t->side[q] && (e = cudaStreamCreateWithFlags(&t->side[q], cudaStreamNonBlocking)) != cudaSuccess) return e;
    if (!t->join_ev[q] && (e = cudaEventCreateWithFlags(&t->join_ev[q], cudaEventDisableTiming)) != cudaSuccess)
      return e;
    if ((e = cudaStreamWaitEvent(t->side[q], t->fork_ev, 0)) != cudaSuccess) return e;
    if ((e = launch_one(fmt_nmono(q) + 1, t->side[q], work0 + q)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(t->join_ev[q], t->side[q])) != cudaSuccess) return e;
  }
  for (int q = 0; q <= FMT_MAX_DEGREE; ++q)
    if ((mask & (1ull << q)) && (e = cudaStreamWaitEvent(s, t->join_ev[q], 0)) != cudaSuccess) return e;
  return cudaSuccess;
}

cudaError_t launch_combine(const fmt_tree* t, int depth, int tree_level, double* R, cudaStream_t s) {
  QRArgs a = make_qr_args(t, depth, R);
  const int64_t n_items = t->lv[depth].n_items;
  if (n_items <= 1) return cudaSuccess;
  cudaError_t e;
  const int mx = t->lv[depth].max_m;
  const QRConfig cfg = qr_config(mx);
  const size_t msm = merge_smem_bytes(mx);
  // Upper tree levels (few pairs in flight): each merge on a cluster of C SMs,
  // C from the estimated pairs of this tree level, raised until a CTA's share
  // of the two triangles fits in shared memory.
  const int64_t est = n_items >> (tree_level + 1);
  if (cfg.merge == 0 && est < 76) {
    int C = est >= 38 ? 2 : est >= 19 ? 4 : 8;
    constexpr int kLW = 8, kW = 32 / kLW;
    while (C < 8 && merge_cl_smem_bytes(mx, C, kW) == 0) C *= 2;
    const size_t csm = merge_cl_smem_bytes(mx, C, kW);
    if (csm > 0) {
      switch (C) {
        case 2: return merge_cl_launch<2, kLW>(a, n_items, csm, tree_level, s);
        case 4: return merge_cl_launch<4, kLW>(a, n_items, csm, tree_level, s);
        default: return merge_cl_launch<8, kLW>(a, n_items, csm, tree_level, s);
      }
    }
  }
  if (cfg.merge == 0 && msm <= 200 * 1024) {
    // Fewer pairs than SMs: the launch asks for more than half of an SM's
    // shared memory, so one CTA fits per SM and no SM runs two merges while
    // others idle (a merge is one CTA's work; the CTAs of the pairs' second
    // items exit at once).
    size_t lsm = msm;
    int dev = 0, nsm = 0, smsm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&smsm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess) {
      const size_t one = (size_t)smsm / 2 + 1024;
      if (est < nsm && one > lsm && one <= 200 * 1024) lsm = one;
    }
    cudaGetLastError();
    if ((e = fmt_smem_at_least((const void*)k_merge, lsm)) != cudaSuccess)
      return e;
    k_merge<<<(unsigned)n_items, kMergeThreads, lsm, s>>>(a, tree_level);
    return cudaGetLastError();
  }
  // the packed triangle does not fit (large degrees) or the configuration
  // asks for row blocks
  const size_t smem = qr_smem_bytes(mx, cfg.rows);
  return qr_ops(cfg).combine(a, (unsigned)n_items, smem, s, tree_level);
}

cudaError_t launch_backsolve(const fmt_tree* t, int depth, double* R, cudaStream_t s) {
  const fmt_level& L = t->lv[depth];
  BSArgs a;
  a.n_nodes = L.n_nodes;
  a.node_item0 = L.node_item0;
  a.R = R;
  a.item_roff = L.item_roff;
  a.depth = depth;
  a.node_prob = L.prob;
  a.prob = t->d_prob;
  a.stride = t->nmono;
  a.ws = backsolve_ws_doubles(L.max_m - 1);
  a.coef = L.coef;
  a.hcoef = L.hcoef;
  a.flags = L.flags;
  a.deg_used = L.deg_used;
  a.n_items = L.n_items;
  a.bd = level_bounds(t, depth);
  const size_t smem = 4 * (size_t)a.ws * sizeof(double);
  cudaError_t e = fmt_smem_at_least((const void*)k_backsolve, smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((L.n_nodes + 3) / 4);
  if (grid == 0) return cudaSuccess;
  k_backsolve<<<grid, 128, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_residual(const fmt_tree* t, int depth, cudaStream_t s, int min_degree) {
  const fmt_level& L = t->lv[depth];
  if (L.n_items <= 0) return cudaSuccess;
  ResArgs a;
  a.item_node = L.item_node;
  a.item_start = L.item_start;
  a.item_end = L.item_end;
  a.prefix = L.prefix;
  a.node_prob = L.prob;
  a.prob = t->d_prob;
  a.x = t->x;
  a.y = t->y;
  a.z = t->z;
  a.r = t->r;
  a.hcoef = L.hcoef;
  a.depth = depth;
  a.stride = t->nmono;
  a.node_start = L.start;
  a.node_count = L.count;
  a.bd = level_bounds(t, depth);
  a.min_degree = min_degree;
  k_residual<<<(unsigned)L.n_items, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_child_stats(const fmt_tree* t, int depth, cudaStream_t s) {
  const fmt_level& L = t->lv[depth];
  if (L.n_nodes <= 0) return cudaSuccess;
  ChildArgs a;
  a.n_nodes = L.n_nodes;
  a.prefix = L.prefix;
  a.start = L.start;
  a.count = L.count;
  a.code = t->code;
  a.r = t->r;
  a.bounds = L.bounds;
  a.child_S = L.child_S;
  a.child_n = L.child_n;
  a.depth = depth;
  a.bd = level_bounds(t, depth);
  const int child_depth = depth + 1;
  a.shift = (child_depth <= FMT_QBITS && child_depth <= t->sort_bits / 3) ? 3 * (FMT_QBITS - child_depth) : -1;
  const int64_t nb = L.n_nodes * 9;
  k_child_bounds<<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(a);
  k_child_sums<<<(unsigned)(L.n_nodes * 8), 128, 0, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free single-node fit (fmt_fit_node_static in include/fmt.h).
//
// Its only scratch, the m x m triangle of the QR (m <= nmono(8) + 1 = 166), is
// this file-scope device array: 166 * 166 doubles = 220,448 bytes, present on
// every GPU that loads the library until the process exits.  All calls on a
// device share it; each call clears the part it uses before the QR starts.
// Host code must not pass the array's name to a kernel (in host code it is a
// stand-in, not a device address): the address is looked up once per device
// with cudaGetSymbolAddress and cached below.
static __device__ __align__(256) double g_static_tri[FMT_STATIC_MAX_M * FMT_STATIC_MAX_M];

namespace {

struct StaticArgs {
  int64_t n;
  const double* x;
  const double* y;
  const double* z;
  const double* r_in;
  double* r_out;
  double* coef;
  int32_t* flags;
  double lo0, lo1, lo2, side, inv_side;
  int p, q, m, ldB, nmono_p;
  double* R;
};

// One CTA: structured Householder over all rows into the static triangle,
// back substitution by warp 0, then the residual update by every thread.
__global__ void __launch_bounds__(kQRThreads) k_fit_node_static(StaticArgs a) {
  extern __shared__ double smem[];
  constexpr int RPT = 16, NB = 4 * RPT;
  double* Bs = smem;
  double* Rs = smem + NB * a.ldB;
  double* sc = Rs + 2 * a.ldB;
  double* G = sc + 4;  // F / (l! m! n!), degree-p layout
  if (!FMT_CHECK(a.q >= -1 && a.q <= a.p && a.p <= FMT_STATIC_MAX_DEGREE && a.m == fmt_nmono_d(a.q) + 1 &&
                     a.m <= FMT_STATIC_MAX_M && a.n >= 0,
                 CK_STATIC_ROWS))
    return;
  const int m = a.m, q = a.q;
  double* R = a.R;
  for (int e = threadIdx.x; e < m * m; e += kQRThreads) {
    const int j = e / m, k = e - j * m;
    if (k >= j) R[e] = 0.0;
  }
  double c0, s0, c1, s1, c2, s2;
  fmt_frame(a.lo0, a.side, a.inv_side, 0, 0u, c0, s0);
  fmt_frame(a.lo1, a.side, a.inv_side, 0, 0u, c1, s1);
  fmt_frame(a.lo2, a.side, a.inv_side, 0, 0u, c2, s2);
  __syncthreads();
  for (int64_t b0 = 0; b0 < a.n; b0 += NB) {
    const int nb = (int)((a.n - b0) < NB ? (a.n - b0) : NB);
    if (threadIdx.x < NB) {
      double* row = Bs + threadIdx.x * a.ldB;
      if ((int)threadIdx.x < nb) {
        const int64_t i = b0 + threadIdx.x;
        const double u = fmt_local(a.x[i], c0, s0), v = fmt_local(a.y[i], c1, s1), w = fmt_local(a.z[i], c2, s2);
        double pu[FMT_MAX_DEGREE + 1], pv[FMT_MAX_DEGREE + 1], pw[FMT_MAX_DEGREE + 1];
        double tu = 1.0, tv = 1.0, tw = 1.0;
        for (int l = 0; l <= q; ++l) {
          const double f = c_invfact[l];
          pu[l] = tu * f;
          pv[l] = tv * f;
          pw[l] = tw * f;
          tu *= u;
          tv *= v;
          tw *= w;
        }
        int k = 0;
        for (int l = 0; l <= q; ++l)
          for (int mm = 0; mm <= q - l; ++mm) {
            const double plm = pu[l] * pv[mm];
            for (int n = 0; n <= q - l - mm; ++n) row[k++] = plm * pw[n];
          }
        row[k] = a.r_in[i];
      } else {
        for (int k = 0; k < m; ++k) row[k] = 0.0;
      }
    }
    __syncthreads();
    absorb_block<RPT, kQRThreads / 32>(Bs, a.ldB, 0, m, R, Rs, sc, -1);
  }
  if ((threadIdx.x >> 5) == 0) {
    const int ndrop = backsolve_warp(R, m, q, a.p, a.nmono_p, Bs, a.coef, G);
    if (threadIdx.x == 0 && a.flags)
      *a.flags = (ndrop > 0 ? FMT_FLAG_RANK : 0) | (q != a.p ? FMT_FLAG_DEG_CLAMPED : 0);
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < a.n; i += kQRThreads) {
    const double u = fmt_local(a.x[i], c0, s0), v = fmt_local(a.y[i], c1, s1), w = fmt_local(a.z[i], c2, s2);
    a.r_out[i] = a.r_in[i] - fmt_horner_t<false>(G, a.p, a.nmono_p, u, v, w);  // G is in shared memory
  }
}

std::mutex g_static_mu;
double* g_static_addr[64];
bool g_static_ready[64];
unsigned long long g_static_ctx[64];  // driver id of the context g_static_addr belongs to (0: unknown)

// The driver's unique id of the device's current context, or 0.  A
// cudaDeviceReset destroys the primary context and the module with it; the
// next runtime call creates a new context with a new id (ids are never
// reused), so a changed id marks the cached symbol address as stale.  The
// driver entry points come through the runtime, so the library does not link
// against libcuda.
unsigned long long current_ctx_id() {
  typedef int (*ctx_get_current_t)(void**);
  typedef int (*ctx_get_id_t)(void*, unsigned long long*);
  static ctx_get_current_t get_current = nullptr;
  static ctx_get_id_t get_id = nullptr;
  static std::once_flag looked_up;
  std::call_once(looked_up, [] {
    void* a = nullptr;
    void* b = nullptr;
    cudaDriverEntryPointQueryResult qa, qb;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
        qa == cudaDriverEntryPointSuccess && qb == cudaDriverEntryPointSuccess) {
      get_current = (ctx_get_current_t)a;
      get_id = (ctx_get_id_t)b;
    }
    cudaGetLastError();
  });
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

}  // namespace

// The largest limit set so far per (context, kernel).  A context id of 0
// (the driver query unavailable) still never lowers a limit: the largest
// value seen for the kernel is set again.
cudaError_t fmt_smem_at_least(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<unsigned long long, const void*>, size_t> lim;
  const unsigned long long ctx = current_ctx_id();
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = lim[std::make_pair(ctx, func)];
  if (ctx != 0 && bytes <= cur) return cudaSuccess;
  const size_t want = bytes > cur ? bytes : cur;
  const cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)want);
  if (e == cudaSuccess) cur = want;
  return e;
}

extern "C" fmt_status fmt_fit_node_static(int32_t degree, int64_t n, const double* x, const double* y,
                                          const double* z, const double* r_in, const double* lo, double side,
                                          double* coef, double* r_out, int32_t* flags, void* stream) {
  char msg[200];
  if (degree < 0 || degree > FMT_STATIC_MAX_DEGREE) {
    snprintf(msg, sizeof(msg),
             "fmt_fit_node_static: degree %d outside [0, %d] (its static triangle holds %d x %d doubles)",
             degree, FMT_STATIC_MAX_DEGREE, FMT_STATIC_MAX_M, FMT_STATIC_MAX_M);
    return fmt_set_error(FMT_EINVAL, msg);
  }
  if (n < 1 || n > (int64_t)0x7fffffff) return fmt_set_error(FMT_EINVAL, "fmt_fit_node_static: n outside [1, 2^31-1]");
  if (!x || !y || !z || !r_in || !lo || !coef || !r_out)
    return fmt_set_error(FMT_EINVAL, "fmt_fit_node_static: NULL pointer argument");
  if (!(side > 0.0) || !isfinite(side) || !isfinite(lo[0]) || !isfinite(lo[1]) || !isfinite(lo[2]))
    return fmt_set_error(FMT_EINVAL, "fmt_fit_node_static: the box needs finite lo and side > 0");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) return fmt_set_error(FMT_ECUDA, "fmt_fit_node_static: no current device");
  double* R = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_static_mu);
    // cudaSetDevice creates the device's primary context if a reset destroyed it
    if ((e = cudaSetDevice(dev)) != cudaSuccess) {
      snprintf(msg, sizeof(msg), "fmt_fit_node_static: cudaSetDevice failed: %s", cudaGetErrorString(e));
      return fmt_set_error(FMT_ECUDA, msg);
    }
    const unsigned long long ctx = current_ctx_id();
    if (!g_static_ready[dev] || ctx == 0 || ctx != g_static_ctx[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_static_tri);
      if (e != cudaSuccess) {
        snprintf(msg, sizeof(msg), "fmt_fit_node_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        return fmt_set_error(FMT_ECUDA, msg);
      }
      g_static_addr[dev] = (double*)ptr;
      g_static_ready[dev] = true;
      g_static_ctx[dev] = current_ctx_id();
    }
    R = g_static_addr[dev];
  }
  int q = degree;
  if (n < fmt_nmono(degree)) {
    q = -1;
    while (fmt_nmono(q + 1) <= n) ++q;
  }
  StaticArgs a;
  a.n = n;
  a.x = x;
  a.y = y;
  a.z = z;
  a.r_in = r_in;
  a.r_out = r_out;
  a.coef = coef;
  a.flags = flags;
  a.lo0 = lo[0];
  a.lo1 = lo[1];
  a.lo2 = lo[2];
  a.side = side;
  a.inv_side = 1.0 / side;
  a.p = degree;
  a.q = q;
  a.m = fmt_nmono(q) + 1;
  a.ldB = ld_for(a.m);
  a.nmono_p = fmt_nmono(degree);
  a.R = R;
  const size_t smem = ((size_t)66 * a.ldB + 4 + a.nmono_p) * sizeof(double);
  e = fmt_smem_at_least((const void*)k_fit_node_static, smem);
  if (e == cudaSuccess) {
    k_fit_node_static<<<1, kQRThreads, smem, (cudaStream_t)stream>>>(a);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "fmt_fit_node_static: launch failed: %s", cudaGetErrorString(e));
    return fmt_set_error(FMT_ECUDA, msg);
  }
  return check_end(nullptr, (cudaStream_t)stream);
}

extern "C" fmt_status fmt_tune_get(int32_t degree, fmt_tune_entry* out) {
  if (!out || degree < 0 || degree > FMT_MAX_DEGREE)
    return fmt_set_error(FMT_EINVAL, "fmt_tune_get: degree outside [0, 14] or NULL output");
  *out = tune_current(degree);
  return FMT_OK;
}

extern "C" fmt_status fmt_tune_set(const fmt_tune_entry* entry) {
  if (!entry) return fmt_set_error(FMT_EINVAL, "fmt_tune_set: NULL entry");
  if (tune_install(*entry) != FMT_OK)
    return fmt_set_error(FMT_EINVAL,
                         "fmt_tune_set: bad entry (degree 0..14, rows 16/32/48/64/128 within 227 KB of shared memory, "
                         "warps 4/8, chunk_factor 1/2/4/8/16, merge 0/1)");
  return FMT_OK;
}

#ifdef FMT_CHECKED
FMT_CHECK_READER(check_site_fit)
#endif
