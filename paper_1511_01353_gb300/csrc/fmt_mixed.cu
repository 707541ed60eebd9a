// fmt_mixed.cu -- the mixed-precision fit of one level (FMT_MIXED).
//
// Alg. 2 asks, per node, for the least-squares fit of the residual r by the
// polynomials of total degree <= p.  The FP64 path factorises [Lambda | r] by
// Householder QR, which costs 2 m^2 FP64 flops per row (m = nmono + 1).  Here
// the same fit is computed with the O(n m^2) part on the tensor cores:
//
//  1. k_mbox: per node, max |u| per axis and max |r| over its points.  The
//     basis is B = P_a(t_x) P_b(t_y) P_c(t_z) (Legendre, a+b+c <= p) with
//     t = 2^e u, e the largest power of two that keeps |t| <= 1; r is scaled
//     by a power of two to O(1).  Same polynomial space as Alg. 2's moments,
//     so the same least-squares function; far better conditioned.
//  2. k_mgram: per work item, the Gram matrix [B | r]^T [B | r] on the tensor
//     cores (tcgen05.mma kind::f16): the basis (in double-float) and r are
//     cut into four fixed-point digits stored as BF16 tiles; the six leading
//     digit-tile products are accumulated in FP32 in tensor memory, and every
//     1024 rows the accumulator is added into a double-float (FP32 pair) copy
//     in global memory; k_mreduce sums a node's items in FP64.
//     The digit tiles are also stored in HBM (TMA bulk stores) for the sweeps.
//  3. k_mfactor: per node, the item Grams are summed in FP64 and factorised by
//     Cholesky; the factor is R-hat = [[R, Q^T r], [0, rho]] of the FP64 path
//     (the same matrix's R factor, up to row signs).  F = R^{-1} Q^T r.
//  4. sweeps: s = r - Lambda F (k_msresid, double-float), g = B^T s on the tensor
//     cores from the stored digit tiles (TMA bulk loads) and the integer
//     digits of s, exactly (k_mgram projection mode), F += R^{-1} R^{-T} g
//     (k_mupdate; the triangular solves on four warps).
//  5. F is converted to the moment basis of Alg. 2 in the node frame (exact
//     in the scaling, Legendre coefficients are dyadic rationals), so the
//     evaluation and the export are those of the FP64 path; the residual
//     update r <- r - Lambda F evaluates it in double-float (k_mresid_final).
// Nodes with fewer than 1.5 m points (nearly square) on a level with few of
// them skip both tiers: their Householder refit starts with the level on a
// side stream (launch_tile_qr mode 3, fmt_api.cu).
// Acceptance, after every sweep: a node is settled (and skipped by the later
// sweeps) once its change at the data is below kConvergedRel of the fit, its
// change anywhere in the node box below kBoxChangeRel of the problem's
// max |f|, and the bias of the quantised basis (a +-2^-31 perturbation solved
// through R^T R) within the same box bound.  A node that fails, or whose
// Cholesky pivot is below kPivotFloor of its diagonal entry, loses
// FMT_FLAG_MIXED.  Nodes of degree 1..10 that did not fail on the pivot (and
// are not a clamped root) then go to the FP64 normal-equations tier (k_dgram,
// k_dfactor, k_dproj, k_dupdate: FP64 Gram, Cholesky and corrected
// semi-normal sweeps, kept only if a rounding-size perturbation moves the
// polynomial by less than the box bound; FMT_FLAG_MIXED_FP64).  Degrees above
// 9 skip the tensor cores, degrees above 10 both tiers.  What neither tier
// keeps is refitted by the Householder kernels of fmt_fit.cu.

#include <cuda_bf16.h>
#include <float.h>

#include "fmt_internal.cuh"

namespace {

constexpr int kAtom = 64;        // rows per operand tile: one 128-byte swizzle row of BF16
constexpr int kDrainAtoms = 4;   // projection: exact FP32 sums, promoted every 256 rows
constexpr int kGramDrainAtoms = 16;  // Gram: FP32 sums (not exact anyway) promoted every 1024 rows
constexpr int kFThreads = 256;   // factor / update kernels
constexpr int kFPanel = 16;      // rows per panel of the factor's Cholesky
constexpr double kPivotFloor = 1e-6;
constexpr double kConvergedRel = 1e-7;
constexpr double kBoxChangeRel = 1e-8;  // remaining change over the node box, relative to max |f| of the problem
constexpr unsigned long long kWaitNs = 2000000000ull;  // bound of every mbarrier wait
constexpr int kMStat = 8;        // per-node words of mstat
constexpr int kSettled = 7;      // mstat word: 1 once the node passed every acceptance test (later sweeps skip it)

// ------------------------------------------------------------------ shapes
__host__ __device__ __forceinline__ int mpad16(int m) { return (m + 15) & ~15; }
// operand-tile rows: an M = 128 MMA reads rows [0, 128) even for small m
__host__ __device__ __forceinline__ int mrows_for(int m) {
  const int l = mpad16(m);
  return l < 128 ? 128 : l;
}
// TMEM columns of the Gram: band 0 = rows [0,128) x cols [0, Lp); band 1 =
// rows [Lp-128, Lp) x cols [128, Lp) when Lp > 128
__host__ __device__ __forceinline__ int gram_cols(int m) {
  const int l = mpad16(m);
  return l <= 128 ? l : l + (l - 128);
}
__host__ __device__ __forceinline__ bool mixed_ok_degree(int p) { return p >= 0 && p <= FMT_MIXED_MAX_DEGREE; }
// (hard: a nearly square node sent straight to Householder, routed_hard)
__device__ __forceinline__ bool mixed_eligible(const fmt_problem& pr, int depth, bool hard) {
  return mixed_ok_degree(pr.degree) && !(depth == 0 && pr.q_root < pr.degree) && !hard;
}
// the FP64 normal-equations tier takes degrees 1..FMT_MIXED_FP64_MAX_DEGREE:
// above that Householder's rank rule on the badly scaled moment basis of
// Alg. 2 drops columns this tier's Legendre basis would keep (a different
// fit); a clamped root stays with Householder too
__device__ __forceinline__ bool tier2_eligible(const fmt_problem& pr, int depth, bool hard) {
  return pr.degree >= 1 && pr.degree <= FMT_MIXED_FP64_MAX_DEGREE && !(depth == 0 && pr.q_root < pr.degree) &&
         !hard;
}

// ------------------------------------------------------------------ PTX
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase of `parity` to complete; false after limit_ns (and,
// should the global timer ever stand still, after limit_ns polls: each takes
// more than a nanosecond).
__device__ __noinline__ bool mbar_wait_for(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  for (unsigned long long it = 0; !mbar_try(bar, parity); ++it)
    if (gtimer() - t0 > limit_ns || it > limit_ns) return false;
  return true;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) { return mbar_wait_for(bar, parity, kWaitNs); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// whole warp
__device__ __forceinline__ void tc_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// D[tmem] (+)= A * B^T, both operands K-major BF16 in shared memory
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
// the mbarrier completes one phase when every MMA issued so far by this thread is done
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  // the registers are valid only after wait::ld; tie them to it
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15])
               :
               : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Bulk (TMA) copies between shared and global memory.  Addresses 16-byte
// aligned, sizes multiples of 16.
__device__ __forceinline__ void bulk_store(void* gdst, const void* ssrc, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(smem_u32(ssrc)),
               "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// the shared-memory sources of every committed store have been read
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// ... of every committed store but the most recent one
__device__ __forceinline__ void bulk_wait_read_but1() {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
// every committed store is complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// load `bytes` into shared memory; the mbarrier's phase completes when they have landed
__device__ __forceinline__ void bulk_load(void* sdst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(sdst)),
      "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle (8-row
// atoms of 128-byte rows, 16-byte chunks XOR-ed with the row index), atoms
// 1024 bytes apart.  Fields: start >> 4 (bits 0-13), leading offset >> 4
// (16-29, unused for this layout), stride offset >> 4 (32-45), descriptor
// version 1 (46), swizzle mode 2 = 128 B (61-63).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// byte offset of element (row j, k) in a K-major 128-byte-swizzled tile of 64 BF16 per row
__device__ __forceinline__ uint32_t sw_off(int j, int k) {
  return (uint32_t)((j >> 3) * 1024 + (j & 7) * 128 + ((((k >> 3) ^ j) & 7) << 4) + ((k & 7) << 1));
}

// Bonnet's recurrence P_{k+1} = a_k t P_k - b_k P_{k-1}, a_k = (2k+1)/(k+1),
// b_k = k/(k+1): the constants as double-float pairs (hi, lo), k = 1..13.
#define FMT_LA(k) ((double)(2 * (k) + 1) / (double)((k) + 1))
#define FMT_LB(k) ((double)(k) / (double)((k) + 1))
#define FMT_DF(v) {(float)(v), (float)((v) - (double)(float)(v))}
#define FMT_LEG(k) {FMT_DF(FMT_LA(k)), FMT_DF(FMT_LB(k))}
static __constant__ float c_leg_ab[FMT_MAX_DEGREE][2][2] = {
    {{0.0f, 0.0f}, {0.0f, 0.0f}}, FMT_LEG(1), FMT_LEG(2),  FMT_LEG(3),  FMT_LEG(4),  FMT_LEG(5),  FMT_LEG(6),
    FMT_LEG(7),                  FMT_LEG(8), FMT_LEG(9),  FMT_LEG(10), FMT_LEG(11), FMT_LEG(12), FMT_LEG(13)};
#undef FMT_LEG
#undef FMT_DF
#undef FMT_LB
#undef FMT_LA

// ------------------------------------------------------------------ node frame
struct MFrame {
  double c[3], s[3], ex[3];  // u = (x - c) s ; t = u ex (ex = 2^e)
  int e[3];
  double sig;                // r scale: sig max|r| in [0.5, 1)
};
__device__ __forceinline__ MFrame mframe(const fmt_problem& pr, uint64_t key, int depth,
                                         const unsigned long long* ms) {
  MFrame F;
  const uint64_t pf = fmt_morton_part(key, depth);
  fmt_frame(pr.lo[0], pr.side, pr.inv_side, depth, fmt_compact3(pf), F.c[0], F.s[0]);
  fmt_frame(pr.lo[1], pr.side, pr.inv_side, depth, fmt_compact3(pf >> 1), F.c[1], F.s[1]);
  fmt_frame(pr.lo[2], pr.side, pr.inv_side, depth, fmt_compact3(pf >> 2), F.c[2], F.s[2]);
  for (int a = 0; a < 3; ++a) {
    const double mu = __longlong_as_double((long long)ms[a]);
    int e = 0;
    while (e < 20 && ldexp(mu, e + 1) <= 1.0) ++e;
    F.e[a] = e;
    F.ex[a] = ldexp(1.0, e);
  }
  const double mr = __longlong_as_double((long long)ms[3]);
  int er = 0;
  if (mr > 0.0) frexp(mr, &er);
  F.sig = ldexp(1.0, -er);
  return F;
}

__device__ __forceinline__ double block_max_d(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double r = 0.0;
  for (int i = 0; i < nw; ++i) r = fmax(r, red[i]);
  return r;
}

// ------------------------------------------------------------------ args
struct MArgs {
  const int64_t* item_node;
  const int64_t* item_start;
  const int64_t* item_end;
  const int32_t* sched;
  const int64_t* node_item0;
  const int32_t* node_nitems;
  int n_items;
  int64_t n_nodes;
  int* work;
  const uint64_t* prefix;
  const int32_t* node_prob;
  const fmt_problem* prob;
  int32_t* flags;
  int32_t* deg_used;
  const double* x;
  const double* y;
  const double* z;
  const double* r;
  double* s;                    // sweep residual, sorted order
  unsigned long long* mstat;    // kMStat per node: max |u|,|v|,|w|, max |r| (bit patterns), last update norm
  double* acc;                  // per item: Gram accumulator (acc_stride doubles) / R-hat of the node
  int64_t acc_stride;
  double* gacc;                 // per item: projection accumulator, 256 doubles
  double* lcoef;                // per node: F in the Legendre basis (stride doubles)
  double* coef;
  double* hcoef;
  int stride;                   // coefficient stride (nmono of the largest degree)
  int depth;
  int MR;                       // operand-tile rows of the level
  int tmem_cols;
  int nstages;                  // operand-tile stages (1 or 2) of k_mgram
  uint8_t* cache;               // projection: digit tiles of every atom (4 tiles, cache_atom_bytes)
  int cache_mode;               // 0 generate, 1 generate and store, 2 load
  uint32_t cache_atom_bytes;
  int last_sweep;
  int* err;
  int tier;                     // sweeps of tier 1 (tensor-core Gram) or tier 2 (FP64 Gram)
  double* rbuf;                 // tier 2: per item the packed FP64 Gram, per node R (first item), in the QR scratch
  const int64_t* item_roff;     // offset of each item's slot in rbuf
  double* dproj;                // tier 2: per item B^T s (dstride doubles)
  int dstride;
  const int64_t* node_start;    // the level's node point ranges (the checked build's tests;
  const int64_t* node_count;    // the count also keeps nearly square nodes off both tiers)
  fmt_bounds bd;
  int route_hard;               // route_hard(): nearly square nodes go straight to Householder
  double* r_out;                // k_mresid_final: the residual, updated in place
};
// a nearly square node this level sends straight to Householder
__device__ __forceinline__ bool routed_hard(const MArgs& a, int64_t node, const fmt_problem& pr) {
  return a.route_hard && fmt_mixed_hard(pr.degree, a.node_count[node]);
}

#ifdef FMT_CHECKED
// Checked build: a node's problem and degree (its coefficients fit the
// stride, its m the level's largest) and its items inside the level's.
__device__ __forceinline__ bool mixed_node_ok(const MArgs& a, int64_t node) {
  if (!fmt_in(node, a.bd.n_nodes) || !fmt_in(a.node_prob[node], a.bd.n_problems)) return false;
  const int p = a.prob[a.node_prob[node]].degree;
  if (p < 0 || p > FMT_MAX_DEGREE || fmt_nmono_d(p) > a.stride || fmt_nmono_d(p) > a.dstride) return false;
  const int64_t i0 = a.node_item0[node], ni = a.node_nitems[node];
  return ni >= 1 && i0 >= 0 && i0 + ni <= a.bd.n_items;
}
// ... and an item of it: the rows inside its node's inside the points.
__device__ __forceinline__ bool mixed_item_ok(const MArgs& a, int64_t item) {
  if (!fmt_in(item, a.bd.n_items)) return false;
  const int64_t node = a.item_node[item];
  if (!mixed_node_ok(a, node)) return false;
  const int64_t s = a.node_start[node], e = s + a.node_count[node];
  const int64_t rs = a.item_start[item], re = a.item_end[item];
  return 0 <= s && s <= rs && rs <= re && re <= e && e <= a.bd.n_points;
}
// The node's m (nmono + 1) within the level's largest, which sized the
// launch's shared memory and accumulators; the FP64 tier also needs each
// item's m x m slot of the QR scratch.
__device__ __forceinline__ bool mixed_m_ok(const MArgs& a, int64_t node, bool slots) {
  const int64_t m = fmt_nmono_d(a.prob[a.node_prob[node]].degree) + 1;
  if (m > a.bd.max_m) return false;
  if (!slots) return true;
  const int64_t i0 = a.node_item0[node], ni = a.node_nitems[node];
  for (int64_t i = i0; i < i0 + ni; ++i) {
    const int64_t ro = a.item_roff[i];
    if (ro < 0 || ro + m * m > a.bd.r_cap) return false;
  }
  return true;
}
#endif
__device__ __forceinline__ bool settled(const MArgs& a, int64_t node) {
  return a.mstat[kMStat * node + kSettled] != 0ull;
}

// ------------------------------------------------------------------ k_mbox
__global__ void __launch_bounds__(256) k_mbox(MArgs a) {
  __shared__ double red[8];
  const int item = blockIdx.x;
  if (!FMT_CHECK(mixed_item_ok(a, item), CK_MIXED_ITEM)) return;
  const int64_t node = a.item_node[item];
  const fmt_problem& pr = a.prob[a.node_prob[node]];
  if (!tier2_eligible(pr, a.depth, routed_hard(a, node, pr))) return;  // the frame serves both tiers
  const uint64_t pf = fmt_morton_part(a.prefix[node], a.depth);
  double c0, s0, c1, s1, c2, s2;
  fmt_frame(pr.lo[0], pr.side, pr.inv_side, a.depth, fmt_compact3(pf), c0, s0);
  fmt_frame(pr.lo[1], pr.side, pr.inv_side, a.depth, fmt_compact3(pf >> 1), c1, s1);
  fmt_frame(pr.lo[2], pr.side, pr.inv_side, a.depth, fmt_compact3(pf >> 2), c2, s2);
  double mu = 0.0, mv = 0.0, mw = 0.0, mr = 0.0;
  for (int64_t i = a.item_start[item] + threadIdx.x; i < a.item_end[item]; i += blockDim.x) {
    mu = fmax(mu, fabs(fmt_local(a.x[i], c0, s0)));
    mv = fmax(mv, fabs(fmt_local(a.y[i], c1, s1)));
    mw = fmax(mw, fabs(fmt_local(a.z[i], c2, s2)));
    mr = fmax(mr, fabs(a.r[i]));
  }
  mu = block_max_d(mu, red);
  mv = block_max_d(mv, red);
  mw = block_max_d(mw, red);
  mr = block_max_d(mr, red);
  if (threadIdx.x == 0) {
    // non-negative doubles order like their bit patterns
    unsigned long long* d = a.mstat + kMStat * node;
    atomicMax(d + 0, (unsigned long long)__double_as_longlong(mu));
    atomicMax(d + 1, (unsigned long long)__double_as_longlong(mv));
    atomicMax(d + 2, (unsigned long long)__double_as_longlong(mw));
    atomicMax(d + 3, (unsigned long long)__double_as_longlong(mr));
  }
}

// ------------------------------------------------------------------ k_mgram
// Both modes store the basis (double-float, pairs of FP32, about 48 bits) as
// the four pre-scaled digit tiles below.  Gram mode: the six leading tile
// products (digit indices q_a + q_b <= 2, a split-BF16 product of about 24
// bits) are accumulated together in FP32 in tensor memory and drained into a
// double-float copy every 1024 rows (not exact: the products' weights differ).
// Projection mode: the basis tiles times the digits of s (FP64), both
// values cut into four signed 8-bit digits of a fixed-point number
// (|P_l(t)| <= 1 for |t| <= 1, and |s| is scaled below 1 per node):
//   v = (d0 2^23 + d1 2^15 + d2 2^7 + d3) 2^-30,   |d| <= 128,
// so every digit is an exact BF16 integer and each digit pair's sum over 256
// rows stays below 2^22: the FP32 tensor-core accumulation is exact, each
// pair has its own accumulator, and the pairs are combined in FP64.

// four signed digits of round(v 2^30), |v| <= 1
__device__ __forceinline__ void digits4(int X, int (&d)[4]) {
  d[0] = (X + (1 << 22)) >> 23;  // arithmetic shifts: floor division
  X -= d[0] * (1 << 23);
  d[1] = (X + (1 << 14)) >> 15;
  X -= d[1] * (1 << 15);
  d[2] = (X + (1 << 6)) >> 7;
  d[3] = X - d[2] * (1 << 7);
}
__host__ __device__ constexpr float digit_scale(int q) {
  return q == 0 ? 0x1p-7f : q == 1 ? 0x1p-15f : q == 2 ? 0x1p-23f : 0x1p-30f;
}
// The basis tiles hold the four digits of round(v 2^30) pre-scaled, d_q 2^e_q
// (exact in BF16), one per tile: the tiles sum to v (to 2^-31), so products
// of tiles carry their weights, and a tile times the integer digits of s
// sums exactly in FP32 over 256 rows (|d| <= 128).
// digits_of: those four digits, pre-scaled, from a double-float |v| <= 1 without
// integer conversions: adding and subtracting 1.5 * 2^(23+e) rounds an FP32
// value to a multiple of 2^e (round to nearest even), and every remainder is
// exact; v.l enters below 2^-8, rounding at 2^-32.  d[q] = d_q 2^e_q.
__device__ __forceinline__ void digits_of(dfl v, float (&d)[4]) {
  d[0] = __fsub_rn(__fadd_rn(v.h, 0x1.8p16f), 0x1.8p16f);     // multiple of 2^-7
  float r = __fadd_rn(__fsub_rn(v.h, d[0]), v.l);
  d[1] = __fsub_rn(__fadd_rn(r, 0x1.8p8f), 0x1.8p8f);         // 2^-15
  r = __fsub_rn(r, d[1]);
  d[2] = __fsub_rn(__fadd_rn(r, 0x1.8p0f), 0x1.8p0f);         // 2^-23
  r = __fsub_rn(r, d[2]);
  d[3] = __fsub_rn(__fadd_rn(r, 0x1.8p-7f), 0x1.8p-7f);       // 2^-30
}
// digits of the points k (even) and k+1 of row j: one 32-bit store per tile
__device__ __forceinline__ void put_digits_f2(uint8_t* t0, uint32_t tile_bytes, int j, int k, const float (&da)[4],
                                              const float (&db)[4]) {
  const uint32_t o = sw_off(j, k);
#pragma unroll
  for (int q = 0; q < 4; ++q)
    *reinterpret_cast<__nv_bfloat162*>(t0 + q * tile_bytes + o) = __floats2bfloat162_rn(da[q], db[q]);
}

// One 64-row atom of the operand tiles is generated in two phases: 192
// threads evaluate the 1-D Legendre values P_0..P_p of the atom's rows (one
// axis each) into shared memory; then every thread takes one row and every
// eighth column j, forms P_l(t_x) P_m(t_y) P_n(t_z) for the (l, m, n) of j and
// stores its BF16 terms / digits.
constexpr int kGThreads = 512;                // 16 warps: 15 generate and drain, the last issues the MMAs
constexpr int kGenThreads = kGThreads - 32;   // generator threads
constexpr int kLegBytes = 3 * (FMT_MIXED_MAX_DEGREE + 1) * kAtom * 8;

// One atom's tensor-core work, handed from the generators to the MMA warp.
struct MmaJob {
  uint32_t A0;  // shared address of the stage
  int N0, Lp, band1, b1;
  int acc;      // 0: the atom opens a drain window (its first MMA overwrites the accumulator)
  int stop;
};

// barrier 1 among the generator warps only
__device__ __forceinline__ void gen_bar() { asm volatile("bar.sync 1, %0;" ::"n"(kGenThreads) : "memory"); }
__device__ __forceinline__ bool gen_bar_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kGenThreads)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// The MMA warp: one job per atom, in order, until a stop job.
template <bool kProj>
__device__ void mma_loop(uint64_t* fbar, uint64_t* mbar, volatile MmaJob* job, int nst, uint32_t tmem,
                         uint32_t tile_bytes, int* err) {
  uint32_t nfull[2] = {0u, 0u};
  int st = 0;
  for (;;) {
    if (!mbar_wait(&fbar[st], nfull[st] & 1u)) {
      atomicOr(err, FMT_ERR_TIMEOUT);
      return;
    }
    nfull[st] += 1u;
    const uint32_t A0 = job[st].A0;
    const int N0 = job[st].N0, Lp = job[st].Lp, b1 = job[st].b1, acc = job[st].acc;
    const bool band1 = job[st].band1 != 0;
    if (job[st].stop) return;
    tc_fence_after();
    if (!kProj) {
      const int pa[6] = {0, 0, 1, 1, 0, 2}, pb[6] = {0, 1, 0, 1, 2, 0};
      const uint32_t id0 = idesc_bf16(128, N0), id1 = band1 ? idesc_bf16(128, Lp - 128) : 0u;
#pragma unroll
      for (int pi = 0; pi < 6; ++pi)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t accf = (acc || pi > 0 || kk > 0) ? 1u : 0u;
          const uint32_t A = A0 + pa[pi] * tile_bytes + 32u * kk, B = A0 + pb[pi] * tile_bytes + 32u * kk;
          tc_mma(tmem, sdesc(A), sdesc(B), id0, accf);
          if (band1) tc_mma(tmem + (uint32_t)N0, sdesc(A + (uint32_t)(b1 >> 3) * 1024u), sdesc(B + 16u * 1024u), id1, accf);
        }
    } else {
      // digit tile q of the basis -> its own accumulators: columns [32 q, 32 q + 16) band 0, +16 band 1
      const uint32_t S = A0 + 4u * tile_bytes;
      const uint32_t id = idesc_bf16(128, 16);
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t accf = (acc || kk > 0) ? 1u : 0u;
          const uint32_t A = A0 + q * tile_bytes + 32u * kk;
          tc_mma(tmem + 32u * q, sdesc(A), sdesc(S + 32u * kk), id, accf);
          if (band1) tc_mma(tmem + 32u * q + 16u, sdesc(A + (uint32_t)(b1 >> 3) * 1024u), sdesc(S + 32u * kk), id, accf);
        }
    }
    tc_commit(&mbar[st]);
    st = (st + 1) % nst;
  }
}

// Persistent over the level's work items (largest first).  Gram mode
// (kProj = false): acc[item] += [B | sig r]^T [B | sig r], column-major by
// TMEM column, 128 lanes each.  Projection mode: gacc[item] += B^T s,
// band 0 rows in [0,128), band 1 rows in [128,256).  Warps 0..14 generate the
// operand tiles of an atom into a free stage and hand it to warp 15, which
// issues its MMAs and commits them to the stage's mbarrier; the generators
// go on with the next atom meanwhile.
template <bool kProj>
__global__ void __launch_bounds__(kGThreads, 1) k_mgram(MArgs a) {
  extern __shared__ uint8_t dsm_raw[];
  __shared__ __align__(8) uint64_t mbar[2];  // the MMAs of a stage are complete
  __shared__ __align__(8) uint64_t fbar[2];  // a stage's job is ready for the MMA warp
  __shared__ __align__(8) uint64_t lbar[2];  // a stage's cached tiles have landed
  __shared__ MmaJob job[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_item, s_deg;
  __shared__ uint16_t s_lmn[(FMT_MIXED_MAX_DEGREE + 1) * (FMT_MIXED_MAX_DEGREE + 2) * (FMT_MIXED_MAX_DEGREE + 3) / 6];
  __shared__ uint16_t s_jb[kGenThreads / 32 + 1];  // column range of each generator warp
  __shared__ double s_val[kAtom];
  constexpr int kTiles = 4;  // the four digit tiles of the basis (Gram: plus the r row)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t* dsm = dsm_raw + ((1024u - (smem_u32(dsm_raw) & 1023u)) & 1023u);
  const uint32_t tile_bytes = (uint32_t)a.MR * 128u;
  const uint32_t stage_bytes = kTiles * tile_bytes + (kProj ? 2048u : 0u);
  const int nst = a.nstages;
  const uint32_t total = (uint32_t)nst * stage_bytes;
  dfl* legd = reinterpret_cast<dfl*>(dsm + total);  // [3][p+1][64] double-float Legendre values
  for (uint32_t o = 16u * tid; o < total; o += 16u * kGThreads) *reinterpret_cast<uint4*>(dsm + o) = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&mbar[i], 1);
      mbar_init(&fbar[i], 1);
      mbar_init(&lbar[i], 1);
    }
    fence_mbar_init();
    s_deg = -1;
  }
  const int cmode = a.cache_mode;  // Gram: 0 or 1 (store the tiles); projection: 0 or 2 (load them)
  if (warp == 0) tc_alloc(&tmem_slot, (uint32_t)a.tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t sbase = smem_u32(dsm);

  if (warp == kGThreads / 32 - 1) {
    if (lane == 0) mma_loop<kProj>(fbar, mbar, job, nst, tmem, tile_bytes, a.err);
    __syncwarp();
  } else {
    uint32_t ncommit[2] = {0u, 0u}, nload[2] = {0u, 0u};
    bool pending[2] = {false, false};
    int hi[2] = {0, 0};  // rows of each stage that may hold non-zero values
    int stage = 0;
    bool ok = true;
    const int k = tid & (kAtom - 1);
    const int lg = warp & 3;               // TMEM lane group of this warp
    const int trow_lane = 32 * lg + lane;  // TMEM lane (matrix row) this thread drains

    for (;;) {
      if (tid == 0) s_item = atomicAdd(a.work, 1);
      gen_bar();
      const int it = s_item;
      gen_bar();
      if (it >= a.n_items) break;
      const int item = a.sched[it];
      // (the generator warps take the same decision)
      if (!FMT_CHECK(mixed_item_ok(a, item), CK_MIXED_ITEM)) continue;
      const int64_t node = a.item_node[item];
      const fmt_problem& pr = a.prob[a.node_prob[node]];
      if (kProj ? (!(a.flags[node] & FMT_FLAG_MIXED) || settled(a, node))
                : !mixed_eligible(pr, a.depth, routed_hard(a, node, pr)))
        continue;
      if (!FMT_CHECK(mixed_m_ok(a, node, false), CK_MIXED_ITEM)) continue;
      const int p = pr.degree;
      const int L = fmt_nmono_d(p), m = L + 1, Lp = mpad16(m);
      const int nw = kProj ? L : m;
      const int N0 = kProj ? 16 : Lp;
      const bool band1 = Lp > 128;
      const int b1 = Lp - 128;
      if (p != s_deg) {  // (l, m, n) of every column, Alg. 2 order
        for (int j = tid; j < L; j += kGenThreads) {
          int r = j, l = 0;
          while (r >= (p - l + 1) * (p - l + 2) / 2) {
            r -= (p - l + 1) * (p - l + 2) / 2;
            ++l;
          }
          int mm = 0;
          while (r >= p - l - mm + 1) {
            r -= p - l - mm + 1;
            ++mm;
          }
          s_lmn[j] = (uint16_t)(l | (mm << 4) | (r << 8));
        }
        gen_bar();
        if (tid == 0) {
          // Contiguous column ranges of about equal work per generator warp:
          // a column costs 4 units (its product and digits), 2 more where
          // its (l, m) differs from the column before (the x-y product is
          // formed again), and the r row (the last warp's) 4.
          constexpr int kW = kGenThreads / 32;
          int total = 4;
          for (int j = 0; j < L; ++j) total += 4 + ((j == 0 || (s_lmn[j] & 255) != (s_lmn[j - 1] & 255)) ? 2 : 0);
          int w = 0, acc = 0;
          s_jb[0] = 0;
          for (int j = 0; j < L && w < kW - 1; ++j) {
            acc += 4 + ((j == 0 || (s_lmn[j] & 255) != (s_lmn[j - 1] & 255)) ? 2 : 0);
            if (acc * kW >= total * (w + 1)) s_jb[++w] = (uint16_t)(j + 1);
          }
          while (w < kW) s_jb[++w] = (uint16_t)L;
          s_deg = p;
        }
        gen_bar();
      }
      const MFrame F = mframe(pr, a.prefix[node], a.depth, a.mstat + kMStat * node);
      // projection: |s| scaled below 1 by a power of two (max |s| of the node, this sweep)
      int se = 0;
      if (kProj) {
        const double ms = __longlong_as_double((long long)a.mstat[kMStat * node + 5]);
        if (ms > 0.0) frexp(ms, &se);
      }
      const double vscale = kProj ? ldexp(1.0, -se) : F.sig;
      const int64_t rs = a.item_start[item], re = a.item_end[item];
      const int natoms = (int)((re - rs + kAtom - 1) / kAtom);
      double* acc = kProj ? a.gacc + (int64_t)item * 256 : a.acc + (int64_t)item * a.acc_stride;
      const double* val = kProj ? a.s : a.r;
      // phase A's operand of the next atom, loaded one atom ahead (a point
      // coordinate for threads 0..191, the value for 192..255)
      const double* pre_src = tid < 3 * kAtom ? (tid < kAtom ? a.x : tid < 2 * kAtom ? a.y : a.z) : val;
      const bool pre_on = (tid < 3 * kAtom && cmode != 2) || (tid >= 3 * kAtom && tid < 4 * kAtom);
      double pre = pre_on && rs + k < re ? pre_src[rs + k] : 0.0;
      bool first_drain = true;
      dfl g0 = {0.0f, 0.0f}, g1 = {0.0f, 0.0f};  // projection, threads < 128: sums of band 0 / 1 at lane tid
      int since = 0;
      for (int at = 0; at < natoms && ok; ++at) {
        const int st = stage;
        if (pending[st]) {
          ok = mbar_wait(&mbar[st], (ncommit[st] - 1u) & 1u);
          pending[st] = false;
        }
        // the stage's previous store (two atoms back with two stages) has read
        // it; the store of the other stage, one atom back, may still be reading
        if (cmode == 1 && tid == 0) {
          if (nst > 1)
            bulk_wait_read_but1();
          else
            bulk_wait_read();
        }
        if (gen_bar_or(!ok)) {
          ok = false;
          break;
        }
        uint8_t* t0 = dsm + st * stage_bytes;
        const int64_t atom_idx = (int64_t)item + (rs >> 6) + at;  // items are disjoint, ascending row ranges
        if (cmode == 2) {
          // the basis digits come from the cache; only s is generated
          if (tid == 0) bulk_load(t0, a.cache + atom_idx * a.cache_atom_bytes, a.cache_atom_bytes, &lbar[st]);
          nload[st] += 1u;
        }
        // rows past this node's basis must read as zero
        if (cmode != 2 && hi[st] > nw) {
          const int nz = (hi[st] - nw) * 8;  // 16-byte words per tile
          for (int e = tid; e < kTiles * nz; e += kGenThreads) {
            const int tt = e / nz, wi = e - tt * nz;
            *reinterpret_cast<uint4*>(t0 + tt * tile_bytes + nw * 128 + wi * 16) = make_uint4(0, 0, 0, 0);
          }
        }
        hi[st] = nw;
        // phase A: 1-D Legendre values (threads 0..191) and the value column (192..255)
        const int64_t i0 = rs + (int64_t)at * kAtom;
        const double cur = pre;
        if (pre_on) pre = i0 + kAtom + k < re ? pre_src[i0 + kAtom + k] : 0.0;
        if (tid < 3 * kAtom && cmode != 2) {
          const int ax = tid / kAtom;
          const int64_t i = i0 + k;
          const double t = i < re ? fmt_local(cur, F.c[ax], F.s[ax]) * F.ex[ax] : 0.0;
          dfl* q = legd + ax * (p + 1) * kAtom + k;
          const dfl td = df_of(t);
          dfl qm = {1.0f, 0.0f}, q0 = td;
          q[0] = qm;
          if (p >= 1) q[kAtom] = q0;
          for (int kk = 1; kk < p; ++kk) {
            const dfl ca = {c_leg_ab[kk][0][0], c_leg_ab[kk][0][1]}, cb = {c_leg_ab[kk][1][0], c_leg_ab[kk][1][1]};
            const dfl qn = df_sub(df_mul(ca, df_mul(td, q0)), df_mul(cb, qm));
            q[(kk + 1) * kAtom] = qn;
            qm = q0;
            q0 = qn;
          }
        } else if (tid >= 3 * kAtom && tid < 4 * kAtom) {
          const int64_t i = i0 + k;
          s_val[k] = i < re ? cur * vscale : 0.0;
        }
        gen_bar();
        // phase B: products as pre-scaled digits; generator warp w takes a
        // contiguous range of columns, lane l the points 2l and 2l+1
        const int P1 = p + 1;
        const int kp = 2 * lane;
        const bool va = i0 + kp < re, vb = i0 + kp + 1 < re;
        if (cmode != 2) {
          const float4* qx = reinterpret_cast<const float4*>(legd + kp);
          const float4* qy = reinterpret_cast<const float4*>(legd + P1 * kAtom + kp);
          const float4* qz = reinterpret_cast<const float4*>(legd + 2 * P1 * kAtom + kp);
          const int jb = s_jb[warp], je = s_jb[warp + 1];
          int plm_key = -1;
          dfl pa = {0.0f, 0.0f}, pb = {0.0f, 0.0f};
          for (int j = jb; j < je; ++j) {
            const int c = s_lmn[j];
            if ((c & 255) != plm_key) {
              plm_key = c & 255;
              const float4 x = qx[(c & 15) * (kAtom / 2)], y = qy[((c >> 4) & 15) * (kAtom / 2)];
              pa = df_mul(dfl{x.x, x.y}, dfl{y.x, y.y});
              pb = df_mul(dfl{x.z, x.w}, dfl{y.z, y.w});
            }
            const float4 z = qz[(c >> 8) * (kAtom / 2)];
            float da[4] = {0.0f, 0.0f, 0.0f, 0.0f}, db[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            if (va) digits_of(df_mul(pa, dfl{z.x, z.y}), da);
            if (vb) digits_of(df_mul(pb, dfl{z.z, z.w}), db);
            put_digits_f2(t0, tile_bytes, j, kp, da, db);
          }
        }
        if (warp == kGenThreads / 32 - 1 || (cmode == 2 && warp == 0)) {
          // |value * vscale| < 1: round(. 2^30) exactly from FP64
          const int Xa = __double2int_rn(s_val[kp] * 1073741824.0), Xb = __double2int_rn(s_val[kp + 1] * 1073741824.0);
          if (!kProj) {
            if (warp == kGenThreads / 32 - 1) {  // r: row L of the tiles
              int ia[4], ib[4];
              digits4(Xa, ia);
              digits4(Xb, ib);
              float da[4], db[4];
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                da[q] = (float)ia[q] * digit_scale(q);
                db[q] = (float)ib[q] * digit_scale(q);
              }
              put_digits_f2(t0, tile_bytes, L, kp, da, db);
            }
          } else if (cmode == 2 ? warp == 0 : warp == kGenThreads / 32 - 1) {
            int ia[4], ib[4];  // s: integer digits, rows 0..3 of the s tile
            digits4(Xa, ia);
            digits4(Xb, ib);
            uint8_t* stile = t0 + 4 * tile_bytes;
#pragma unroll
            for (int q = 0; q < 4; ++q)
              *reinterpret_cast<__nv_bfloat162*>(stile + sw_off(q, kp)) =
                  __floats2bfloat162_rn((float)ia[q], (float)ib[q]);
          }
        }
        fence_async_smem();
        if (cmode == 2 && tid == 0 && !mbar_wait(&lbar[st], (nload[st] - 1u) & 1u)) ok = false;
        gen_bar();
        if (tid == 0) {
          job[st].A0 = sbase + (uint32_t)st * stage_bytes;
          job[st].N0 = N0;
          job[st].Lp = Lp;
          job[st].band1 = band1 ? 1 : 0;
          job[st].b1 = b1;
          job[st].acc = since > 0 ? 1 : 0;
          job[st].stop = 0;
          mbar_arrive(&fbar[st]);
          if (cmode == 1) bulk_store(a.cache + atom_idx * a.cache_atom_bytes, t0, a.cache_atom_bytes);
        }
        ncommit[st] += 1u;
        pending[st] = true;
        stage = (stage + 1) % nst;
        ++since;
        if (since == (kProj ? kDrainAtoms : kGramDrainAtoms) || at == natoms - 1) {
          for (int s2 = 0; s2 < 2; ++s2)
            if (pending[s2]) {
              ok = mbar_wait(&mbar[s2], (ncommit[s2] - 1u) & 1u) && ok;
              pending[s2] = false;
            }
          if (gen_bar_or(!ok)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t trow = tmem + ((uint32_t)(32 * lg) << 16);
          if (!kProj) {
            // the first 4 kDrainGroups generator warps: kDrainGroups per lane
            // group, every kDrainGroups-th 16-column chunk
            constexpr int kDrainGroups = (kGenThreads / 32) / 4;
            if (warp < 4 * kDrainGroups) {
              // double-float running sums on the FP32 pipe (k_mreduce turns them into FP64)
              const int ncols = band1 ? N0 + (Lp - 128) : N0;
              float2* acc2 = reinterpret_cast<float2*>(acc);
              for (int c0 = 16 * (warp >> 2); c0 < ncols; c0 += 16 * kDrainGroups) {
                float vv[16];
                tc_ld16(trow + (uint32_t)c0, vv);
                float2* dst = acc2 + (int64_t)c0 * 128 + trow_lane;
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                  if (first_drain) {
                    dst[q * 128] = make_float2(vv[q], 0.0f);
                  } else {
                    const float2 o = dst[q * 128];
                    const dfl r = df_add(dfl{o.x, o.y}, dfl{vv[q], 0.0f});
                    dst[q * 128] = make_float2(r.h, r.l);
                  }
                }
              }
            }
          } else if (warp < 4) {
            // exact integer sums per (basis tile, s digit), weighted in FP64
            // each term (an FP32 integer sum times 2^e_c) is exact in FP32; the
            // running sums are double-float (warp w < 4 drains lanes 32w.., thread tid = lane)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              float vv[16];
              tc_ld16(trow + 32u * q, vv);
#pragma unroll
              for (int c = 0; c < 4; ++c) g0 = df_add(g0, dfl{vv[c] * digit_scale(c), 0.0f});
              if (band1) {
                tc_ld16(trow + 32u * q + 16u, vv);
#pragma unroll
                for (int c = 0; c < 4; ++c) g1 = df_add(g1, dfl{vv[c] * digit_scale(c), 0.0f});
              }
            }
          }
          first_drain = false;
          since = 0;
          tc_fence_before();
          gen_bar();
        }
      }
      if (!ok) break;
      if (kProj && tid < 128) {
        // B^T s of this item: undo the scale of s
        acc[tid] = ldexp((double)g0.h + (double)g0.l, se);
        if (band1) acc[128 + tid] = ldexp((double)g1.h + (double)g1.l, se);
      }
    }
    // stop the MMA warp (after the job last handed over on that stage is done)
    const int st = stage;
    if (pending[st]) mbar_wait(&mbar[st], (ncommit[st] - 1u) & 1u);
    for (int s2 = 0; s2 < 2; ++s2)
      if (pending[s2]) {
        ok = mbar_wait(&mbar[s2], (ncommit[s2] - 1u) & 1u) && ok;
        pending[s2] = false;
      }
    if (tid == 0) {
      if (!ok) atomicOr(a.err, FMT_ERR_TIMEOUT);
      job[st].stop = 1;
      mbar_arrive(&fbar[st]);
      if (cmode == 1) bulk_wait_all();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tc_dealloc(tmem, (uint32_t)a.tmem_cols);
  }
}

// ------------------------------------------------------------------ change of basis
// Fl (shared, L values, Alg. 2 index order over (a,b,c)) holds the fit in the
// basis P_a(2^ex u) P_b(2^ey v) P_c(2^ez w); writes the same polynomial in the
// moment basis u^l v^m w^n / (l! m! n!) (coef) and its Horner form (hcoef).
// ws: shared scratch of 4 (p+1)^2 doubles + (p+1)^2 ints.
__device__ void legendre_to_moments(const double* Fl, int p, const MFrame& F, double* coef, double* hcoef,
                                    int stride, double* ws) {
  const int P1 = p + 1;
  double* C = ws;  // C[a][l][k] = coefficient of u^k in P_l(2^e_a u)
  int* base = reinterpret_cast<int*>(ws + 3 * P1 * P1);  // index of (l, m, 0)
  for (int e = threadIdx.x; e < 3 * P1 * P1; e += blockDim.x) {
    const int ax = e / (P1 * P1), rem = e - ax * P1 * P1, l = rem / P1, kk = rem - l * P1;
    double v = 0.0;
    if (kk <= l && ((l - kk) & 1) == 0) {
      // P_l(t) = 2^-l sum_j (-1)^j C(l,j) C(2l-2j, l) t^(l-2j)
      const int j = (l - kk) / 2;
      long long c1 = 1, c2 = 1;
      for (int i = 1; i <= j; ++i) c1 = c1 * (l - j + i) / i;
      for (int i = 1; i <= l; ++i) c2 = c2 * (2 * l - 2 * j - l + i) / i;
      v = ldexp((double)(c1 * c2), -l);
      if (j & 1) v = -v;
      v = ldexp(v, F.e[ax] * kk);  // t^k = 2^(e k) u^k
    }
    C[e] = v;
  }
  if (threadIdx.x == 0) {
    int idx = 0;
    for (int l = 0; l <= p; ++l)
      for (int mm = 0; mm <= p - l; ++mm) {
        base[l * P1 + mm] = idx;
        idx += p - l - mm + 1;
      }
  }
  __syncthreads();
  const double* Cx = C;
  const double* Cy = C + P1 * P1;
  const double* Cz = C + 2 * P1 * P1;
  const int L = fmt_nmono_d(p);
  for (int J = threadIdx.x; J < L; J += blockDim.x) {
    int l = 0, mm = 0;
    while (l < p && base[(l + 1) * P1] <= J) ++l;
    while (mm < p - l && base[l * P1 + mm + 1] <= J) ++mm;
    const int n = J - base[l * P1 + mm];
    double h = 0.0;
    for (int l2 = l; l2 <= p; l2 += 2)
      for (int m2 = mm; m2 <= p - l2; m2 += 2) {
        const double cxy = Cx[l2 * P1 + l] * Cy[m2 * P1 + mm];
        const int b = base[l2 * P1 + m2];
        for (int n2 = n; n2 <= p - l2 - m2; n2 += 2) h = fma(Fl[b + n2] * cxy, Cz[n2 * P1 + n], h);
      }
    hcoef[J] = h;
    // F_lmn multiplies u^l v^m w^n / (l! m! n!)
    double f = h;
    for (int i = 2; i <= l; ++i) f *= (double)i;
    for (int i = 2; i <= mm; ++i) f *= (double)i;
    for (int i = 2; i <= n; ++i) f *= (double)i;
    coef[J] = f;
  }
  for (int J = L + threadIdx.x; J < stride; J += blockDim.x) {
    coef[J] = 0.0;
    hcoef[J] = 0.0;
  }
  __syncthreads();
}

__host__ __device__ __forceinline__ int64_t ro_of(int i, int m) { return (int64_t)i * m - (int64_t)i * (i - 1) / 2; }
__host__ __device__ __forceinline__ int conv_ws_doubles(int p) { return 4 * (p + 1) * (p + 1) + 2; }

// ------------------------------------------------------------------ k_mreduce
// Sums the Gram accumulators of a node's work items ((hi, lo) FP32 pairs)
// in FP64 into its first item's accumulator (fixed item order:
// deterministic).  Grid: nodes x chunks of kRedChunk accumulator words, so a
// root split into hundreds of items is reduced by many SMs.
constexpr int kRedChunk = 256;
__global__ void __launch_bounds__(256) k_mreduce(MArgs a, int chunks) {
  const int64_t node = blockIdx.x / chunks;
  const int ch = blockIdx.x - (int)(node * chunks);
  if (!FMT_CHECK(mixed_node_ok(a, node), CK_MIXED_NODE)) return;
  const int ni = a.node_nitems[node];
  const fmt_problem& pr = a.prob[a.node_prob[node]];
  if (!mixed_eligible(pr, a.depth, routed_hard(a, node, pr))) return;
  if (!FMT_CHECK(mixed_m_ok(a, node, false), CK_MIXED_NODE)) return;
  const int64_t words = (int64_t)gram_cols(fmt_nmono_d(pr.degree) + 1) * 128;
  const int64_t i0 = a.node_item0[node];
  // the Gram kernel leaves (hi, lo) FP32 pairs; the node's sum goes to its first item as FP64
  for (int64_t e = (int64_t)ch * kRedChunk + threadIdx.x; e < words && e < (int64_t)(ch + 1) * kRedChunk;
       e += blockDim.x) {
    double sum = 0.0;
    for (int t = 0; t < ni; ++t) {
      const float2 v = reinterpret_cast<const float2*>(a.acc + (i0 + t) * a.acc_stride)[e];
      sum += (double)v.x + (double)v.y;
    }
    a.acc[i0 * a.acc_stride + e] = sum;
  }
}

// ------------------------------------------------------------------ k_mfactor
// One CTA per node.  Shared: the packed upper triangle of the m x m Gram
// (row i at ro(i), m = nmono + 1 with r last), the initial diagonal, y, F and
// the change-of-basis scratch.
// Triangular solves with R packed upper (row i at ro_of(i, m), entry j >= i
// at offset j - i) and invd = 1 / R_ii, by the first kSolveThreads threads of
// the CTA (four warps, one per SM sub-partition): at each step every thread
// updates at most two entries, so a step costs about one FP64 instruction
// per sub-partition instead of one warp's several.  The steps are ordered by
// named barrier 1 (those threads only).
constexpr int kSolveThreads = 128;
__device__ __forceinline__ void solve_bar() { asm volatile("bar.sync 1, %0;" ::"n"(kSolveThreads) : "memory"); }

// Two unknowns per barrier: every thread forms both from shared memory (the
// second one after the first one's term), then updates its entries with both.
// R^T w = g (w overwrites g); returns |w|^2 in thread 0.
__device__ double cta_fwd_solve(const double* __restrict__ R, int m, int L, const double* __restrict__ invd,
                                double* __restrict__ g) {
  const int t = threadIdx.x;
  double wn = 0.0;
  int k = 0;
  for (; k + 1 < L; k += 2) {
    const double* r0 = R + ro_of(k, m) - k;          // r0[j] = R[k][j]
    const double* r1 = R + ro_of(k + 1, m) - (k + 1);  // r1[j] = R[k+1][j]
    const double w0 = g[k] * invd[k];
    const double w1 = fma(-r0[k + 1], w0, g[k + 1]) * invd[k + 1];
    for (int j = k + 2 + t; j < L; j += kSolveThreads) g[j] = fma(-r1[j], w1, fma(-r0[j], w0, g[j]));
    if (t == 0) wn = fma(w1, w1, fma(w0, w0, wn));
    solve_bar();  // g[k + 2] is final; every thread has read g[k], g[k + 1]
    if (t == 0) {
      g[k] = w0;
      g[k + 1] = w1;
    }
  }
  if (k < L) {
    const double w0 = g[k] * invd[k];
    if (t == 0) wn = fma(w0, w0, wn);
    solve_bar();
    if (t == 0) g[k] = w0;
  }
  solve_bar();
  return wn;
}

// R x = y (x overwrites y).
__device__ void cta_back_solve(const double* __restrict__ R, int m, int L, const double* __restrict__ invd,
                               double* __restrict__ y) {
  const int t = threadIdx.x;
  int j = L - 1;
  for (; j >= 1; j -= 2) {
    const double x0 = y[j] * invd[j];
    const double x1 = fma(-R[ro_of(j - 1, m) + 1], x0, y[j - 1]) * invd[j - 1];  // R[j-1][j]
    for (int i = t; i < j - 1; i += kSolveThreads) {
      const double* ri = R + ro_of(i, m) - i;  // ri[c] = R[i][c]
      y[i] = fma(-ri[j - 1], x1, fma(-ri[j], x0, y[i]));
    }
    solve_bar();  // y[j - 2] is final; every thread has read y[j], y[j - 1]
    if (t == 0) {
      y[j] = x0;
      y[j - 1] = x1;
    }
  }
  if (j == 0) {
    const double x0 = y[0] * invd[0];
    solve_bar();
    if (t == 0) y[0] = x0;
  }
  solve_bar();
}

__global__ void __launch_bounds__(kFThreads) k_mfactor(MArgs a) {
  extern __shared__ double fsm[];
  const int64_t node = blockIdx.x;
  if (!FMT_CHECK(mixed_node_ok(a, node), CK_MIXED_NODE)) return;
  const fmt_problem& pr = a.prob[a.node_prob[node]];
  if (!mixed_eligible(pr, a.depth, routed_hard(a, node, pr))) return;
  if (!FMT_CHECK(mixed_m_ok(a, node, false), CK_MIXED_NODE)) return;
  const int tid = threadIdx.x;
  const int p = pr.degree, L = fmt_nmono_d(p), m = L + 1, Lp = mpad16(m), b1 = Lp - 128;
  const int ncols = gram_cols(m);
  // Shared: G | rk | invd | Fl (114.9 KB at degree 8, so two CTAs fit on an
  // SM); the change of basis at the end reuses G, rk and invd, and the pivot
  // test reads the Gram's diagonal from global memory (thread 0 only).
  double* G = fsm;
  double* rk = G + ro_of(m, m);
  double* invd = rk + m;
  double* Fl = invd + m;
  double* ws = G;
  const int64_t i0 = a.node_item0[node];
  const double* Gg = a.acc + i0 * a.acc_stride;  // the summed Gram, band layout (column c, lane i)
  auto diag0 = [&](int k) {  // G[k][k] before the factorisation
    return Gg[k < 128 ? (int64_t)k * 129 : (int64_t)(Lp + k - 128) * 128 + (k - b1)];
  };
  // 1. the node's FP64 Gram (column c, lane i), summed over items by k_mreduce
  for (int e = tid; e < ncols * 128; e += kFThreads) {
    const int c = e >> 7, lane = e & 127;
    int gi, gj;
    if (c < Lp) {
      gi = lane;
      gj = c;
      if (gi >= 128) continue;
    } else {
      gi = b1 + lane;
      gj = 128 + (c - Lp);
      if (gi < 128) continue;
    }
    if (gi > gj || gj >= m) continue;
    G[ro_of(gi, m) + (gj - gi)] = a.acc[i0 * a.acc_stride + e];
  }
  // 2. Cholesky on the packed rows, column L (r) carried along, in panels of
  // kFPanel rows: within a panel, column by column, thread 0 forms the pivot
  // (the floor test, one reciprocal square root), the row is scaled and the
  // panel's later rows are updated; then the trailing triangle (rows and
  // columns past the panel) takes the panel's rank-kFPanel update at once,
  // each thread a 4 x 4 register tile (two barriers per panel instead of two
  // per column, and full-warp FMAs).
  __shared__ double s_rkk, s_irk;
  __shared__ int s_bad;
  double d0_next = tid == 0 ? diag0(0) : 0.0;  // thread 0: the next pivot's original diagonal, loaded ahead
  auto pivot = [&](int k) {  // thread 0
    const double d = G[ro_of(k, m)], d0 = d0_next;
    if (k + 1 < L) d0_next = diag0(k + 1);
    s_bad = !(d0 > 0.0 && d > kPivotFloor * d0);
    if (!s_bad) {
      const double ir = rsqrt(d);
      s_irk = ir;
      s_rkk = d * ir;
    }
  };
  __syncthreads();
  for (int k0 = 0; k0 < L; k0 += kFPanel) {
    const int k1 = k0 + kFPanel < L ? k0 + kFPanel : L;
    for (int k = k0; k < k1; ++k) {
      if (tid == 0) pivot(k);
      __syncthreads();
      if (s_bad) {  // the same decision in every thread
        if (tid == 0) {
          a.flags[node] |= FMT_FLAG_MIXED_PIVOT;
          atomicAdd(a.work + kPivSlot, 1);  // the level's count of small-pivot nodes
        }
        return;  // the FP64 path refits this node
      }
      const double rkk = s_rkk, irk = s_irk;
      double* Gk = G + ro_of(k, m) - k;  // Gk[j] = G[k][j]
      for (int j = k + 1 + tid; j < m; j += kFThreads) Gk[j] *= irk;
      if (tid == 0) invd[k] = irk;
      __syncthreads();
      if (tid == 0) Gk[k] = rkk;  // every thread has read the pivot by now
      // the panel's later rows i in (k, k1): G[i][j] -= R[k][i] R[k][j], j >= i
      const int w = m - k - 1;
      for (int e = tid; e < (k1 - k - 1) * w; e += kFThreads) {
        const int i = k + 1 + e / w, j = k + 1 + e % w;
        if (j >= i) G[ro_of(i, m) + (j - i)] = fma(-Gk[i], Gk[j], G[ro_of(i, m) + (j - i)]);
      }
      __syncthreads();
    }
    // trailing triangle, rows and columns in [k1, m): G[i][j] -= sum_{k in panel} R[k][i] R[k][j]
    const int n = m - k1, nt = (n + 3) >> 2, ntiles = nt * (nt + 1) / 2;
    for (int t = tid; t < ntiles; t += kFThreads) {
      int ta = 0, rem = t;  // tile (ta, tb), tb >= ta, row-major over the upper tiles
      while (rem >= nt - ta) {
        rem -= nt - ta;
        ++ta;
      }
      const int tb = ta + rem;
      const int i0 = k1 + 4 * ta, j0 = k1 + 4 * tb;
      double acc[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
      for (int k = k0; k < k1; ++k) {
        const double* Gk = G + ro_of(k, m) - k;
        double ri[4], rj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          ri[u] = i0 + u < m ? Gk[i0 + u] : 0.0;
          rj[u] = j0 + u < m ? Gk[j0 + u] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = fma(ri[u], rj[v], acc[u][v]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int i = i0 + u, j = j0 + v;
          if (i < m && j < m && j >= i) G[ro_of(i, m) + (j - i)] -= acc[u][v];
        }
    }
    __syncthreads();
  }
  // 3. R F = y, y = the scaled Q^T r column
  for (int k = tid; k < L; k += kFThreads) Fl[k] = G[ro_of(k, m) + (L - k)];
  __syncthreads();
  if (tid < kSolveThreads) cta_back_solve(G, m, L, invd, Fl);
  __syncthreads();
  const MFrame F = mframe(pr, a.prefix[node], a.depth, a.mstat + kMStat * node);
  for (int k = tid; k < L; k += kFThreads) {
    Fl[k] = Fl[k] / F.sig;
    a.lcoef[node * a.stride + k] = Fl[k];
  }
  // keep R-hat for the sweeps in the node's first accumulator (the Gram there
  // has been read for the last time: every pivot test is done)
  __syncthreads();
  double* Rg = a.acc + i0 * a.acc_stride;
  for (int64_t e = tid; e < ro_of(m, m); e += kFThreads) Rg[e] = G[e];
  __syncthreads();
  legendre_to_moments(Fl, p, F, a.coef + node * a.stride, a.hcoef + node * a.stride, a.stride, ws);
  if (tid == 0) {
    a.flags[node] |= FMT_FLAG_MIXED;
    a.deg_used[node] = p;
  }
}

// ------------------------------------------------------------------ sweeps
// The node polynomial of fmt_horner_t in double-float with the Horner
// coefficients in shared memory (hi, lo pairs).
__device__ __forceinline__ dfl horner_df_shared(const float2* G, int p, int nmono, dfl u, dfl v, dfl w) {
  int idx = nmono - 1;
  dfl P = {0.0f, 0.0f};
  for (int l = p; l >= 0; --l) {
    dfl t = {0.0f, 0.0f};
    for (int m = p - l; m >= 0; --m) {
      dfl s = {0.0f, 0.0f};
      for (int n = p - l - m; n >= 0; --n) {
        const float2 g = G[idx--];
        s = df_fma(s, w, dfl{g.x, g.y});
      }
      t = df_fma(t, v, s);
    }
    P = df_fma(P, u, t);
  }
  return P;
}

// s = r - Lambda F (the residual of the current fit, r untouched).  The
// tensor-core tier (kDF) evaluates the polynomial in double-float (FP32
// pairs, about 48 bits) on the FP32 pipe, node frame and the final
// subtraction in FP64: the sweeps' fixed point then carries a relative error
// of about 2^-48 of |Lambda F| in s, far below the tier's acceptance bounds
// (1e-7 of the fit, 1e-8 max|f|, and the 2^-31 quantisation of its basis).
// The FP64 tier keeps the FP64 residual its rounding test assumes.
template <bool kDF>
__global__ void __launch_bounds__(256) k_msresid(MArgs a) {
  const int item = blockIdx.x;
  if (!FMT_CHECK(mixed_item_ok(a, item), CK_MIXED_ITEM)) return;
  const int64_t node = a.item_node[item];
  const int32_t nf = a.flags[node];
  if (!(nf & FMT_FLAG_MIXED) || (a.tier == 2 && !(nf & FMT_FLAG_MIXED_FP64)) || settled(a, node)) return;
  const fmt_problem& pr = a.prob[a.node_prob[node]];
  const uint64_t pf = fmt_morton_part(a.prefix[node], a.depth);
  double c0, s0, c1, s1, c2, s2;
  fmt_frame(pr.lo[0], pr.side, pr.inv_side, a.depth, fmt_compact3(pf), c0, s0);
  fmt_frame(pr.lo[1], pr.side, pr.inv_side, a.depth, fmt_compact3(pf >> 1), c1, s1);
  fmt_frame(pr.lo[2], pr.side, pr.inv_side, a.depth, fmt_compact3(pf >> 2), c2, s2);
  const int p = pr.degree, nm = fmt_nmono_d(p);
  const double* Gc = a.hcoef + node * a.stride;
  __shared__ float2 hdf[kDF ? (FMT_MIXED_MAX_DEGREE + 1) * (FMT_MIXED_MAX_DEGREE + 2) * (FMT_MIXED_MAX_DEGREE + 3) / 6 : 1];
  if (kDF) {
    for (int k = threadIdx.x; k < nm; k += blockDim.x) {
      const double g = Gc[k];
      const float h = __double2float_rn(g);
      hdf[k] = make_float2(h, __double2float_rn(g - (double)h));
    }
    __syncthreads();
  }
  double ms = 0.0;
  // each thread's next point is loaded while it evaluates the current one
  const int64_t ie = a.item_end[item];
  int64_t i = a.item_start[item] + threadIdx.x;
  double nx = 0.0, ny = 0.0, nz = 0.0, nr = 0.0;
  if (i < ie) {
    nx = a.x[i];
    ny = a.y[i];
    nz = a.z[i];
    nr = a.r[i];
  }
  for (; i < ie; i += blockDim.x) {
    const double xv = nx, yv = ny, zv = nz, rv = nr;
    if (i + blockDim.x < ie) {
      nx = a.x[i + blockDim.x];
      ny = a.y[i + blockDim.x];
      nz = a.z[i + blockDim.x];
      nr = a.r[i + blockDim.x];
    }
    const double u = fmt_local(xv, c0, s0), v = fmt_local(yv, c1, s1), w = fmt_local(zv, c2, s2);
    double si;
    if (kDF) {
      const dfl P = horner_df_shared(hdf, p, nm, df_of(u), df_of(v), df_of(w));
      si = rv - ((double)P.h + (double)P.l);
    } else {
      si = rv - fmt_horner(Gc, p, nm, u, v, w);
    }
    a.s[i] = si;
    ms = fmax(ms, fabs(si));
  }
  __shared__ double red[8];
  ms = block_max_d(ms, red);
  if (threadIdx.x == 0)
    atomicMax(a.mstat + kMStat * node + 5, (unsigned long long)__double_as_longlong(ms));
}

// The residual update r <- r - Lambda F that ends a level of a mixed tree,
// for the nodes of degree <= FMT_MIXED_MAX_DEGREE, whatever fitted them: the
// polynomial in double-float as in the sweeps (an error of about 2^-48
// |Lambda F|, far below the mixed bar and below the FP64 bar of the nodes
// Householder fitted), frame and subtraction in FP64.  Nodes of higher
// degree keep the FP64 residual (k_residual).
__global__ void __launch_bounds__(256) k_mresid_final(MArgs a) {
  const int item = blockIdx.x;
  if (!FMT_CHECK(mixed_item_ok(a, item), CK_MIXED_ITEM)) return;
  const int64_t node = a.item_node[item];
  const fmt_problem& pr = a.prob[a.node_prob[node]];
  const int p = pr.degree, nm = fmt_nmono_d(p);
  if (p > FMT_MIXED_MAX_DEGREE) return;
  const uint64_t pf = fmt_morton_part(a.prefix[node], a.depth);
  double c0, s0, c1, s1, c2, s2;
  fmt_frame(pr.lo[0], pr.side, pr.inv_side, a.depth, fmt_compact3(pf), c0, s0);
  fmt_frame(pr.lo[1], pr.side, pr.inv_side, a.depth, fmt_compact3(pf >> 1), c1, s1);
  fmt_frame(pr.lo[2], pr.side, pr.inv_side, a.depth, fmt_compact3(pf >> 2), c2, s2);
  const double* Gc = a.hcoef + node * a.stride;
  __shared__ float2 hdf[(FMT_MIXED_MAX_DEGREE + 1) * (FMT_MIXED_MAX_DEGREE + 2) * (FMT_MIXED_MAX_DEGREE + 3) / 6];
  for (int k = threadIdx.x; k < nm; k += blockDim.x) {
    const double g = Gc[k];
    const float h = __double2float_rn(g);
    hdf[k] = make_float2(h, __double2float_rn(g - (double)h));
  }
  __syncthreads();
  const int64_t ie = a.item_end[item];
  int64_t i = a.item_start[item] + threadIdx.x;
  double nx = 0.0, ny = 0.0, nz = 0.0, nr = 0.0;  // the next point, loaded ahead
  if (i < ie) {
    nx = a.x[i];
    ny = a.y[i];
    nz = a.z[i];
    nr = a.r_out[i];
  }
  for (; i < ie; i += blockDim.x) {
    const double xv = nx, yv = ny, zv = nz, rv = nr;
    if (i + blockDim.x < ie) {
      nx = a.x[i + blockDim.x];
      ny = a.y[i + blockDim.x];
      nz = a.z[i + blockDim.x];
      nr = a.r_out[i + blockDim.x];
    }
    const dfl P = horner_df_shared(hdf, p, nm, df_of(fmt_local(xv, c0, s0)), df_of(fmt_local(yv, c1, s1)),
                                   df_of(fmt_local(zv, c2, s2)));
    a.r_out[i] = rv - ((double)P.h + (double)P.l);
  }
}

// F += R^{-1} R^{-T} g per node; on the last sweep a node whose update is
// still above kConvergedRel of its fit loses FMT_FLAG_MIXED.
__global__ void __launch_bounds__(kFThreads) k_mupdate(MArgs a) {
  extern __shared__ double usm[];
  __shared__ double red[kFThreads / 32];
  const int64_t node = blockIdx.x;
  if (!FMT_CHECK(mixed_node_ok(a, node), CK_MIXED_NODE)) return;
  if (!(a.flags[node] & FMT_FLAG_MIXED) || settled(a, node)) return;
  if (!FMT_CHECK(mixed_m_ok(a, node, false), CK_MIXED_NODE)) return;
  const int tid = threadIdx.x;
  const fmt_problem& pr = a.prob[a.node_prob[node]];
  const int p = pr.degree, L = fmt_nmono_d(p), m = L + 1, Lp = mpad16(m), b1 = Lp - 128;
  const MFrame F = mframe(pr, a.prefix[node], a.depth, a.mstat + kMStat * node);
  const int64_t i0 = a.node_item0[node];
  const int ni = a.node_nitems[node];
  // Shared: R | g | invd | Fl (114.9 KB at degree 8: two CTAs per SM); the
  // change of basis at the end reuses R, g and invd, which are dead by then.
  double* R = usm;  // R-hat rows 0..L-1, packed (row i at ro(i)), copied from the node's first accumulator
  double* g = R + ro_of(m, m);
  double* invd = g + m;
  double* Fl = invd + m;
  double* ws = R;
  {
    const double* Rg = a.acc + i0 * a.acc_stride;
    for (int64_t e = tid; e < ro_of(m, m); e += kFThreads) R[e] = Rg[e];
  }
  for (int j = tid; j < L; j += kFThreads) {
    const int e = j < 128 ? j : 128 + (j - b1);
    double sum = 0.0;
    for (int t = 0; t < ni; ++t) sum += a.gacc[(i0 + t) * 256 + e];
    g[j] = sum;  // the projection kernel has undone the scale of s
    Fl[j] = a.lcoef[node * a.stride + j];
  }
  __syncthreads();  // R, g and F complete
  for (int k = tid; k < L; k += kFThreads) invd[k] = 1.0 / R[ro_of(k, m)];
  __syncthreads();
  double wn = 0.0;
  if (tid < kSolveThreads) {
    // |R d|^2 = |R^{-T} g|^2 is taken between the two triangular solves
    wn = cta_fwd_solve(R, m, L, invd, g);
    cta_back_solve(R, m, L, invd, g);
  }
  __syncthreads();
  for (int j = tid; j < L; j += kFThreads) {
    Fl[j] += g[j];
    a.lcoef[node * a.stride + j] = Fl[j];
  }
  __syncthreads();
  // |R F| (the fit at the data) and, over the node box, a bound of the change
  // of the polynomial: |P_a(t_x) P_b(t_y) P_c(t_z)| <= P_a(T_x) P_b(T_y) P_c(T_z)
  // with T = 2^e >= 1 (|u| <= 1 maps to |t| <= T), so the change anywhere in
  // the box is at most sum_j |d_j| P(T)_j
  __shared__ double s_pt[3][FMT_MIXED_MAX_DEGREE + 1];
  if (tid < 3) {
    const double T = F.ex[tid];
    double q0 = 1.0, q1 = T;
    s_pt[tid][0] = 1.0;
    if (p >= 1) s_pt[tid][1] = T;
    for (int kk = 1; kk < p; ++kk) {
      const double q2 = ((double)(2 * kk + 1) * T * q1 - (double)kk * q0) / (double)(kk + 1);
      s_pt[tid][kk + 1] = q2;
      q0 = q1;
      q1 = q2;
    }
  }
  __syncthreads();
  double zn = 0.0, cw = 0.0;
  for (int i = tid; i < L; i += kFThreads) {
    const double* rowi = R + ro_of(i, m) - i;
    double zi = 0.0;
    for (int j = i; j < L; ++j) zi = fma(rowi[j], Fl[j], zi);
    zn += zi * zi;
    // (a, b, c) of column i in Alg. 2 order
    int r = i, la = 0;
    while (r >= (p - la + 1) * (p - la + 2) / 2) {
      r -= (p - la + 1) * (p - la + 2) / 2;
      ++la;
    }
    int lb = 0;
    while (r >= p - la - lb + 1) {
      r -= p - la - lb + 1;
      ++lb;
    }
    cw += fabs(g[i]) * s_pt[0][la] * s_pt[1][lb] * s_pt[2][r];
  }
  for (int o = 16; o > 0; o >>= 1) {
    zn += __shfl_xor_sync(0xffffffffu, zn, o);
    cw += __shfl_xor_sync(0xffffffffu, cw, o);
  }
  __shared__ double red2[kFThreads / 32];
  if ((tid & 31) == 0) {
    red[tid >> 5] = zn;
    red2[tid >> 5] = cw;
  }
  __syncthreads();
  double ztot = 0.0, ctot = 0.0;
  for (int i = 0; i < kFThreads / 32; ++i) {
    ztot += red[i];
    ctot += red2[i];
  }
  // The acceptance tests, after every sweep: the change of the fit at the
  // data |R d| = |Lambda d| against |R F|, and the bound ctot of the change
  // over the node box against kBoxChangeRel max |f| (with the previous
  // sweep's values: the contraction rho and the remaining error ~ change *
  // rho / (1 - rho)).  A node that passes them and the bias test below is
  // settled: the later sweeps skip it.  On the last sweep a node that has not
  // settled goes to the FP64 tier.
  __shared__ int s_conv;
  const double cthr = kBoxChangeRel * pr.maxabs;
  if (tid == 0) {
    unsigned long long* slot = a.mstat + kMStat * node + 4;
    unsigned long long* cslot = a.mstat + kMStat * node + 6;
    const double upd = sqrt(wn), zr = sqrt(ztot), prev = __longlong_as_double((long long)*slot);
    const double cprev = __longlong_as_double((long long)*cslot);
    *slot = (unsigned long long)__double_as_longlong(upd);
    *cslot = (unsigned long long)__double_as_longlong(ctot);
    a.mstat[kMStat * node + 5] = 0ull;  // max |s| of the next sweep
    bool conv = upd <= kConvergedRel * zr;
    if (!conv && prev > 0.0 && upd < prev) {
      const double rho = upd / prev;
      conv = upd * rho / (1.0 - rho) <= kConvergedRel * zr;
    }
    bool cconv = ctot <= cthr;
    if (!cconv && cprev > 0.0 && ctot < cprev) {
      const double rho = ctot / cprev;
      cconv = ctot * rho / (1.0 - rho) <= cthr;
    }
    s_conv = conv && cconv;
  }
  __syncthreads();
  // Bias of the quantised basis: the fixed point solves B~^T (r - Lambda F) = 0
  // with the basis quantised to 2^-31 (the digit tiles), which moves F by
  // (R^T R)^{-1} E^T r_LS, |E_ij| <= 2^-31: about 2^-31 |r_LS| per column.
  // That perturbation (with pseudo-random signs, twice the size) is solved
  // through R^T R and bounded over the box.  |r_LS| = sqrt(R_LL^2) / sig
  // (column L carries sig r).
  const bool check = s_conv || a.last_sweep;
  double etot = 0.0;
  if (check) {
    const double rls = sqrt(fmax(R[ro_of(L, m)], 0.0)) / F.sig;
    const double scale = 2.0 * 0x1p-31 * rls;
    for (int j = tid; j < L; j += kFThreads)
      g[j] = (((uint32_t)j * 2654435761u) >> 16) & 1u ? scale : -scale;
    __syncthreads();
    if (tid < kSolveThreads) {
      cta_fwd_solve(R, m, L, invd, g);
      cta_back_solve(R, m, L, invd, g);
    }
    __syncthreads();
    double ew = 0.0;
    for (int i = tid; i < L; i += kFThreads) {
      int r = i, la = 0;
      while (r >= (p - la + 1) * (p - la + 2) / 2) {
        r -= (p - la + 1) * (p - la + 2) / 2;
        ++la;
      }
      int lb = 0;
      while (r >= p - la - lb + 1) {
        r -= p - la - lb + 1;
        ++lb;
      }
      ew += fabs(g[i]) * s_pt[0][la] * s_pt[1][lb] * s_pt[2][r];
    }
    for (int o = 16; o > 0; o >>= 1) ew += __shfl_xor_sync(0xffffffffu, ew, o);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = ew;
    __syncthreads();
    for (int i = 0; i < kFThreads / 32; ++i) etot += red[i];
  }
  legendre_to_moments(Fl, p, F, a.coef + node * a.stride, a.hcoef + node * a.stride, a.stride, ws);
  if (tid == 0) {
    if (s_conv && etot <= cthr)
      a.mstat[kMStat * node + kSettled] = 1ull;
    else if (a.last_sweep)
      a.flags[node] = (a.flags[node] & ~FMT_FLAG_MIXED) | FMT_FLAG_MIXED_SLOW;
  }
}

// ------------------------------------------------------------------ tier 2
// Nodes the tensor-core tier could not fit (a small pivot, no convergence, or
// a degree above FMT_MIXED_MAX_DEGREE) are fitted by corrected semi-normal
// equations in FP64 before any falls back to Householder: the Gram of
// [B | sig r] in FP64 on the FP64 pipe (n m^2 flops against Householder's
// 2 n m^2), its Cholesky factor, F = R^{-1} R^{-T} B^T r, then sweeps
// F += R^{-1} R^{-T} B^T (r - Lambda F) with the FP64 residual and an FP64
// projection, under the convergence tests of the tensor-core tier.  The basis
// is the same Legendre product basis in the same node frame.  The fixed point
// of the sweeps solves B^T (r - B F) = 0 as evaluated in FP64, whose rounding
// (about c eps |B| (|B| |F| + |r|) in the residual) moves F by up to
// (B^T B)^{-1} of its projection: with a small residual and cancelling
// coefficients (nearly square or clustered nodes) that is kappa times worse
// than Householder.  So after the last sweep a perturbation of that size,
// delta g_j = +-c eps sqrt(G_jj) (sum_k |F_k| sqrt(G_kk) + |r|) with
// pseudo-random signs, is solved through R^T R, and the node is kept only if
// the resulting change of the polynomial over its box stays within
// kRoundRel max |f| (else Householder, which the mixed path is held to,
// refits it).
constexpr double kPivotFloor2 = 1e-12;  // FP64 Gram: a column must keep 1e-6 of its norm
constexpr double kRoundRel = 1e-8;      // bound of the rounding-driven change over the box, relative to max |f|
constexpr int kDT = 64;                 // Gram tile (columns)
constexpr int kDRows = 32;              // rows per shared-memory chunk
constexpr int kPanel = 32;              // rows per Cholesky panel
constexpr int kRT = 4;                  // factored rows staged per update pass

#define FMT_LA64(k) ((double)(2 * (k) + 1) / (double)((k) + 1))
#define FMT_LB64(k) ((double)(k) / (double)((k) + 1))
#define FMT_L64(k) {FMT_LA64(k), FMT_LB64(k)}
// Bonnet's recurrence constants a_k, b_k in FP64, k = 0..13
static __constant__ double c_leg64[FMT_MAX_DEGREE][2] = {
    FMT_L64(0), FMT_L64(1), FMT_L64(2), FMT_L64(3),  FMT_L64(4),  FMT_L64(5),  FMT_L64(6),
    FMT_L64(7), FMT_L64(8), FMT_L64(9), FMT_L64(10), FMT_L64(11), FMT_L64(12), FMT_L64(13)};
#undef FMT_L64
#undef FMT_LB64
#undef FMT_LA64

// A node whose tensor-core Cholesky met a pivot below kPivotFloor is too
// ill-conditioned for the normal equations at the mixed path's bar as well
// (the FP64 tier's rounding check rejects nearly all of them), so it goes to
// Householder directly; the FP64 tier takes the nodes that did not converge
// and those of degree above FMT_MIXED_MAX_DEGREE.
__device__ __forceinline__ bool tier2_selected(const MArgs& a, int64_t node, const fmt_problem& pr) {
  const int32_t f = a.flags[node];
  return tier2_eligible(pr, a.depth, routed_hard(a, node, pr)) && !(f & (FMT_FLAG_MIXED | FMT_FLAG_MIXED_PIVOT));
}

// (a, b, c) of basis column j in Alg. 2 order, packed a | b << 8 | c << 16
__device__ __forceinline__ int col_abc(int j, int p) {
  int r = j, la = 0;
  while (r >= (p - la + 1) * (p - la + 2) / 2) {
    r -= (p - la + 1) * (p - la + 2) / 2;
    ++la;
  }
  int lb = 0;
  while (r >= p - la - lb + 1) {
    r -= p - la - lb + 1;
    ++lb;
  }
  return la | (lb << 8) | (r << 16);
}

// P_0..P_p of one coordinate (FP64 recurrence): t = u 2^e
__device__ __forceinline__ void legendre64(double t, int p, double* P) {
  P[0] = 1.0;
  if (p >= 1) P[1] = t;
  for (int k = 1; k < p; ++k) P[k + 1] = fma(c_leg64[k][0] * t, P[k], -c_leg64[k][1] * P[k - 1]);
}

// The 1-D Legendre values of a chunk of rows: Pl[row][axis][0..p]
__device__ __forceinline__ void chunk_legendre(const MArgs& a, const MFrame& F, int64_t r0, int nr, int p,
                                               double* Pl) {
  constexpr int P1 = FMT_MAX_DEGREE + 1;
  const int tid = threadIdx.x;
  if (tid < 3 * kDRows) {
    const int row = tid / 3, ax = tid - 3 * row;
    double* P = Pl + (row * 3 + ax) * P1;
    if (row < nr) {
      const double* X = ax == 0 ? a.x : ax == 1 ? a.y : a.z;
      const double t = fmt_local(X[r0 + row], F.c[ax], F.s[ax]) * F.ex[ax];
      legendre64(t, p, P);
    } else {
      for (int k = 0; k <= p; ++k) P[k] = 0.0;
    }
  }
}

// Packed upper triangle of one item's FP64 Gram, one 64 x 64 tile (bi, bj)
// per CTA, rows streamed through shared memory 32 at a time.  The tile is
// four 32 x 32 sub-tiles of two warps each (64 threads, 4 x 4 entries per
// thread at rows ty + 8 i, columns tx + 8 j); a sub-tile below the diagonal
// or past column m is skipped by whole warps (at degree 10, 90% of the
// multiply-adds are then entries of the triangle, against 67% for whole tiles).
__global__ void __launch_bounds__(256) k_dgram(MArgs a, int npairs) {
  constexpr int P1 = FMT_MAX_DEGREE + 1;
  __shared__ double Pl[kDRows * 3 * P1];
  __shared__ double As[kDRows][kDT], Bs[kDRows][kDT];
  __shared__ int cabc[2][kDT];
  const int item = blockIdx.x / npairs, pair = blockIdx.x - item * npairs;
  if (!FMT_CHECK(mixed_item_ok(a, item), CK_MIXED_ITEM)) return;
  const int64_t node = a.item_node[item];
  const fmt_problem& pr = a.prob[a.node_prob[node]];
  if (!tier2_selected(a, node, pr)) return;
  if (!FMT_CHECK(mixed_m_ok(a, node, true), CK_MIXED_ITEM)) return;
  const int p = pr.degree, L = fmt_nmono_d(p), m = L + 1, nt = (m + kDT - 1) / kDT;
  if (pair >= nt * (nt + 1) / 2) return;
  int bi = 0, rem = pair;
  while (rem >= nt - bi) {
    rem -= nt - bi;
    ++bi;
  }
  const int bj = bi + rem;
  const bool diag = bi == bj;
  const int tid = threadIdx.x, sub = tid >> 6, sr = sub >> 1, sc = sub & 1;
  const int tx = tid & 7, ty = (tid >> 3) & 7;
  const int ro = bi * kDT + 32 * sr, co = bj * kDT + 32 * sc;     // the sub-tile's first row / column
  const bool active = !(diag && sr > sc) && ro < m && co < m;      // warp-uniform
  const MFrame F = mframe(pr, a.prefix[node], a.depth, a.mstat + kMStat * node);
  if (tid < 2 * kDT) {
    const int w = tid / kDT, c = tid - w * kDT, j = (w ? bj : bi) * kDT + c;
    cabc[w][c] = j < L ? col_abc(j, p) : -1 - (j == L);  // -2: the value column, -1: padding
  }
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  const int64_t rs = a.item_start[item], re = a.item_end[item];
  for (int64_t r0 = rs; r0 < re; r0 += kDRows) {
    const int nr = (int)(re - r0 < kDRows ? re - r0 : kDRows);
    __syncthreads();  // the previous chunk's tiles are consumed
    chunk_legendre(a, F, r0, nr, p, Pl);
    __syncthreads();
    for (int e = tid; e < (diag ? 1 : 2) * kDRows * kDT; e += 256) {
      const int w = e / (kDRows * kDT), r2 = e - w * (kDRows * kDT), row = r2 / kDT, c = r2 - row * kDT;
      const int code = cabc[w][c];
      double v = 0.0;
      if (row < nr) {
        if (code >= 0) {
          const double* P = Pl + row * 3 * P1;
          v = P[code & 0xff] * P[P1 + ((code >> 8) & 0xff)] * P[2 * P1 + (code >> 16)];
        } else if (code == -2) {
          v = a.r[r0 + row] * F.sig;
        }
      }
      (w ? Bs : As)[row][c] = v;
    }
    __syncthreads();
    const double(*Bt)[kDT] = diag ? As : Bs;
    if (active) {
      for (int row = 0; row < nr; ++row) {
        double av[4], bv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          av[i] = As[row][32 * sr + ty + 8 * i];
          bv[i] = Bt[row][32 * sc + tx + 8 * i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
      }
    }
  }
  if (!active) return;
  double* G = a.rbuf + a.item_roff[item];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gi = ro + ty + 8 * i, gj = co + tx + 8 * j;
      if (gi <= gj && gj < m) G[ro_of(gi, m) + (gj - gi)] = acc[i][j];
    }
}

// Per node: the item Grams summed (fixed order) and factorised by a blocked
// left-looking Cholesky, 32-row panels in shared memory; R (packed, column L
// = the scaled R^{-T} B^T r, then rho) overwrites the first item's slot, whose
// rows below the current panel are still the Gram's.  Then F = R^{-1} y.
__global__ void __launch_bounds__(256) k_dfactor(MArgs a) {
  extern __shared__ double dsm[];
  const int64_t node = blockIdx.x;
  if (!FMT_CHECK(mixed_node_ok(a, node), CK_MIXED_NODE)) return;
  const fmt_problem& pr = a.prob[a.node_prob[node]];
  if (!tier2_selected(a, node, pr)) return;
  if (!FMT_CHECK(mixed_m_ok(a, node, true), CK_MIXED_NODE)) return;
  const int tid = threadIdx.x;
  const int p = pr.degree, L = fmt_nmono_d(p), m = L + 1;
  const int64_t i0 = a.node_item0[node];
  const int ni = a.node_nitems[node];
  double* PS = dsm;                  // kPanel rows x m (absolute column index)
  double* RT = PS + kPanel * m;      // kRT factored rows x m
  double* d0 = RT + kRT * m;         // the Gram's diagonal
  double* invd = d0 + m;
  double* Fl = invd + m;
  double* ws = Fl + m;
  __shared__ int s_fail;
  __shared__ double s_piv[2];
  if (tid == 0) s_fail = 0;
  double* R = a.rbuf + a.item_roff[i0];
  for (int k0 = 0; k0 < m; k0 += kPanel) {
    const int k1 = k0 + kPanel < m ? k0 + kPanel : m, np = k1 - k0, w = m - k0;
    __syncthreads();
    for (int e = tid; e < np * w; e += 256) {
      const int r = e / w, j = k0 + (e - r * w), i = k0 + r;
      double v = 0.0;
      if (j >= i) {
        const int64_t o = ro_of(i, m) + (j - i);
        for (int t = 0; t < ni; ++t) v += a.rbuf[a.item_roff[i0 + t] + o];
      }
      PS[r * m + j] = v;
      if (j == i) d0[i] = v;
    }
    // left-looking update by the factored rows t < k0
    for (int t0 = 0; t0 < k0; t0 += kRT) {
      const int nt = k0 - t0 < kRT ? k0 - t0 : kRT;
      __syncthreads();
      for (int e = tid; e < nt * w; e += 256) {
        const int tt = e / w, j = k0 + (e - tt * w), t = t0 + tt;
        RT[tt * m + j] = R[ro_of(t, m) + (j - t)];
      }
      __syncthreads();
      for (int e = tid; e < np * w; e += 256) {
        const int r = e / w, j = k0 + (e - r * w), i = k0 + r;
        if (j < i) continue;
        double v = PS[r * m + j];
        for (int tt = 0; tt < nt; ++tt) v = fma(-RT[tt * m + i], RT[tt * m + j], v);
        PS[r * m + j] = v;
      }
    }
    // the panel itself, right-looking (thread 0 forms each pivot's square
    // root and reciprocal once: FP64 sqrt and divide in every warp are costly)
    for (int k = k0; k < k1 && k < L; ++k) {
      __syncthreads();
      if (tid == 0) {
        const double d = PS[(k - k0) * m + k];
        const bool bad = !(d0[k] > 0.0 && d > kPivotFloor2 * d0[k]);
        s_fail = bad ? 1 : 0;
        if (!bad) {
          s_piv[0] = sqrt(d);
          s_piv[1] = 1.0 / s_piv[0];
        }
      }
      __syncthreads();
      if (s_fail) break;  // the same decision in every thread
      const double rkk = s_piv[0], irk = s_piv[1];
      double* rowk = PS + (k - k0) * m;
      for (int j = k + 1 + tid; j < m; j += 256) rowk[j] *= irk;
      __syncthreads();
      if (tid == 0) {
        rowk[k] = rkk;
        invd[k] = irk;
      }
      const int wk = m - k - 1;
      for (int e = tid; e < (k1 - k - 1) * wk; e += 256) {
        const int r = e / wk, j = k + 1 + (e - r * wk), i = k + 1 + r;
        if (j >= i) PS[(i - k0) * m + j] = fma(-rowk[i], rowk[j], PS[(i - k0) * m + j]);
      }
    }
    __syncthreads();
    if (s_fail) break;
    for (int e = tid; e < np * w; e += 256) {
      const int r = e / w, j = k0 + (e - r * w), i = k0 + r;
      if (j >= i) R[ro_of(i, m) + (j - i)] = PS[r * m + j];
    }
  }
  __syncthreads();
  if (s_fail) {
    if (tid == 0) a.flags[node] |= FMT_FLAG_MIXED_PIVOT;
    return;  // Householder refits this node
  }
  for (int k = tid; k < L; k += 256) Fl[k] = R[ro_of(k, m) + (L - k)];
  for (int k = tid; k < m; k += 256) R[ro_of(m, m) + k] = d0[k];  // the Gram's diagonal, after R (slot of m^2)
  __syncthreads();
  if (tid < kSolveThreads) cta_back_solve(R, m, L, invd, Fl);
  __syncthreads();
  const MFrame F = mframe(pr, a.prefix[node], a.depth, a.mstat + kMStat * node);
  for (int k = tid; k < L; k += 256) {
    Fl[k] = Fl[k] / F.sig;
    a.lcoef[node * a.stride + k] = Fl[k];
  }
  if (tid == 0) {  // convergence history of this tier's sweeps
    a.mstat[kMStat * node + 4] = 0ull;
    a.mstat[kMStat * node + 5] = 0ull;
    a.mstat[kMStat * node + 6] = 0ull;
    a.mstat[kMStat * node + kSettled] = 0ull;
  }
  __syncthreads();
  legendre_to_moments(Fl, p, F, a.coef + node * a.stride, a.hcoef + node * a.stride, a.stride, ws);
  if (tid == 0) {
    a.flags[node] |= FMT_FLAG_MIXED | FMT_FLAG_MIXED_FP64;
    a.deg_used[node] = p;
  }
}

// Per item: B^T s in FP64, one column per thread (three for degree > 8)
__global__ void __launch_bounds__(256) k_dproj(MArgs a) {
  constexpr int P1 = FMT_MAX_DEGREE + 1;
  __shared__ double Pl[kDRows * 3 * P1];
  __shared__ double sv[kDRows];
  const int item = blockIdx.x;
  if (!FMT_CHECK(mixed_item_ok(a, item), CK_MIXED_ITEM)) return;
  const int64_t node = a.item_node[item];
  if ((a.flags[node] & (FMT_FLAG_MIXED | FMT_FLAG_MIXED_FP64)) != (FMT_FLAG_MIXED | FMT_FLAG_MIXED_FP64) ||
      settled(a, node))
    return;
  const fmt_problem& pr = a.prob[a.node_prob[node]];
  const int p = pr.degree, L = fmt_nmono_d(p);
  const int tid = threadIdx.x;
  const MFrame F = mframe(pr, a.prefix[node], a.depth, a.mstat + kMStat * node);
  int code[3];
  double acc[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int q = 0; q < 3; ++q) code[q] = tid + 256 * q < L ? col_abc(tid + 256 * q, p) : -1;
  const int64_t rs = a.item_start[item], re = a.item_end[item];
  for (int64_t r0 = rs; r0 < re; r0 += kDRows) {
    const int nr = (int)(re - r0 < kDRows ? re - r0 : kDRows);
    __syncthreads();
    chunk_legendre(a, F, r0, nr, p, Pl);
    if (tid < kDRows) sv[tid] = tid < nr ? a.s[r0 + tid] : 0.0;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (code[q] < 0) continue;
      const int ca = code[q] & 0xff, cb = P1 + ((code[q] >> 8) & 0xff), cc = 2 * P1 + (code[q] >> 16);
      double g = acc[q];
      for (int row = 0; row < nr; ++row) {
        const double* P = Pl + row * 3 * P1;
        g = fma(P[ca] * P[cb] * P[cc], sv[row], g);
      }
      acc[q] = g;
    }
  }
#pragma unroll
  for (int q = 0; q < 3; ++q)
    if (code[q] >= 0) a.dproj[(int64_t)item * a.dstride + tid + 256 * q] = acc[q];
}

// Per node: F += R^{-1} R^{-T} g with R in global memory (the node's first
// item slot), then the convergence tests of k_mupdate.
__global__ void __launch_bounds__(kFThreads) k_dupdate(MArgs a) {
  extern __shared__ double usm2[];
  __shared__ double red[kFThreads / 32], red2[kFThreads / 32];
  __shared__ double s_pt[3][FMT_MAX_DEGREE + 1];
  const int64_t node = blockIdx.x;
  if (!FMT_CHECK(mixed_node_ok(a, node), CK_MIXED_NODE)) return;
  if ((a.flags[node] & (FMT_FLAG_MIXED | FMT_FLAG_MIXED_FP64)) != (FMT_FLAG_MIXED | FMT_FLAG_MIXED_FP64) ||
      settled(a, node))
    return;
  if (!FMT_CHECK(mixed_m_ok(a, node, true), CK_MIXED_NODE)) return;
  const int tid = threadIdx.x;
  const fmt_problem& pr = a.prob[a.node_prob[node]];
  const int p = pr.degree, L = fmt_nmono_d(p), m = L + 1;
  const MFrame F = mframe(pr, a.prefix[node], a.depth, a.mstat + kMStat * node);
  const int64_t i0 = a.node_item0[node];
  const int ni = a.node_nitems[node];
  const double* R = a.rbuf + a.item_roff[i0];
  double* g = usm2;
  double* Fl = g + m;
  double* invd = Fl + m;
  double* ws = invd + m;
  for (int j = tid; j < L; j += kFThreads) {
    double sum = 0.0;
    for (int t = 0; t < ni; ++t) sum += a.dproj[(i0 + t) * a.dstride + j];
    g[j] = sum;
    Fl[j] = a.lcoef[node * a.stride + j];
    invd[j] = 1.0 / R[ro_of(j, m)];
  }
  __syncthreads();
  double wn = 0.0;
  if (tid < kSolveThreads) {
    wn = cta_fwd_solve(R, m, L, invd, g);  // R^T w = g, then |w|^2 = |R d|^2
    cta_back_solve(R, m, L, invd, g);
  }
  __syncthreads();
  for (int j = tid; j < L; j += kFThreads) {
    Fl[j] += g[j];
    a.lcoef[node * a.stride + j] = Fl[j];
  }
  if (tid < 3) {
    const double T = F.ex[tid];
    double q0 = 1.0, q1 = T;
    s_pt[tid][0] = 1.0;
    if (p >= 1) s_pt[tid][1] = T;
    for (int kk = 1; kk < p; ++kk) {
      const double q2 = ((double)(2 * kk + 1) * T * q1 - (double)kk * q0) / (double)(kk + 1);
      s_pt[tid][kk + 1] = q2;
      q0 = q1;
      q1 = q2;
    }
  }
  __syncthreads();
  const double* d0 = R + ro_of(m, m);  // the Gram's diagonal (k_dfactor)
  double zn = 0.0, cw = 0.0, fa = 0.0;
  for (int i = tid; i < L; i += kFThreads) {
    const double* rowi = R + ro_of(i, m) - i;
    double zi = 0.0;
    for (int j = i; j < L; ++j) zi = fma(rowi[j], Fl[j], zi);
    zn += zi * zi;
    const int c = col_abc(i, p);
    cw += fabs(g[i]) * s_pt[0][c & 0xff] * s_pt[1][(c >> 8) & 0xff] * s_pt[2][c >> 16];
    fa += fabs(Fl[i]) * sqrt(d0[i]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    zn += __shfl_xor_sync(0xffffffffu, zn, o);
    cw += __shfl_xor_sync(0xffffffffu, cw, o);
    fa += __shfl_xor_sync(0xffffffffu, fa, o);
  }
  __shared__ double red3[kFThreads / 32];
  if ((tid & 31) == 0) {
    red[tid >> 5] = zn;
    red2[tid >> 5] = cw;
    red3[tid >> 5] = fa;
  }
  __syncthreads();
  double ztot = 0.0, ctot = 0.0, atot = 0.0;
  for (int i = 0; i < kFThreads / 32; ++i) {
    ztot += red[i];
    ctot += red2[i];
    atot += red3[i];
  }
  // the acceptance tests after every sweep (as in k_mupdate); a node that
  // passes them and the rounding test is settled, later sweeps skip it
  __shared__ int s_conv;
  const double cthr = kBoxChangeRel * pr.maxabs;
  if (tid == 0) {
    unsigned long long* slot = a.mstat + kMStat * node + 4;
    unsigned long long* cslot = a.mstat + kMStat * node + 6;
    const double upd = sqrt(wn), zr = sqrt(ztot), prev = __longlong_as_double((long long)*slot);
    const double cprev = __longlong_as_double((long long)*cslot);
    *slot = (unsigned long long)__double_as_longlong(upd);
    *cslot = (unsigned long long)__double_as_longlong(ctot);
    a.mstat[kMStat * node + 5] = 0ull;
    bool conv = upd <= kConvergedRel * zr;
    if (!conv && prev > 0.0 && upd < prev) {
      const double rho = upd / prev;
      conv = upd * rho / (1.0 - rho) <= kConvergedRel * zr;
    }
    bool cconv = ctot <= cthr;
    if (!cconv && cprev > 0.0 && ctot < cprev) {
      const double rho = ctot / cprev;
      cconv = ctot * rho / (1.0 - rho) <= cthr;
    }
    s_conv = conv && cconv;
  }
  __syncthreads();
  // the rounding perturbation of the fixed point, solved through R^T R
  double etot = 0.0;
  if (s_conv || a.last_sweep) {
    const double rn = sqrt(d0[L]) / F.sig;  // |r|: column L of the Gram is sig r
    const double scale = (double)(3 * p + 4) * DBL_EPSILON * (atot + rn);
    for (int j = tid; j < L; j += kFThreads) {
      const uint32_t hsh = (uint32_t)j * 2654435761u;
      g[j] = ((hsh >> 16) & 1u ? scale : -scale) * sqrt(d0[j]);
    }
    __syncthreads();
    if (tid < kSolveThreads) {
      cta_fwd_solve(R, m, L, invd, g);
      cta_back_solve(R, m, L, invd, g);
    }
    __syncthreads();
    double ew = 0.0;
    for (int i = tid; i < L; i += kFThreads) {
      const int c = col_abc(i, p);
      ew += fabs(g[i]) * s_pt[0][c & 0xff] * s_pt[1][(c >> 8) & 0xff] * s_pt[2][c >> 16];
    }
    for (int o = 16; o > 0; o >>= 1) ew += __shfl_xor_sync(0xffffffffu, ew, o);
    __syncthreads();
    if ((tid & 31) == 0) red3[tid >> 5] = ew;
    __syncthreads();
    for (int i = 0; i < kFThreads / 32; ++i) etot += red3[i];
  }
  legendre_to_moments(Fl, p, F, a.coef + node * a.stride, a.hcoef + node * a.stride, a.stride, ws);
  if (tid == 0) {
    if (s_conv && etot <= kRoundRel * pr.maxabs)  // insensitive to the FP64 rounding
      a.mstat[kMStat * node + kSettled] = 1ull;
    else if (a.last_sweep)
      a.flags[node] = (a.flags[node] & ~(FMT_FLAG_MIXED | FMT_FLAG_MIXED_FP64)) | FMT_FLAG_MIXED_SLOW;
  }
}

int nsm() {
  static const int n = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  return n;
}

MArgs make_margs(const fmt_tree* t, int depth, const fmt_mixed_bufs& b) {
  const fmt_level& L = t->lv[depth];
  MArgs a;
  a.item_node = L.item_node;
  a.item_start = L.item_start;
  a.item_end = L.item_end;
  a.sched = L.sched;
  a.node_item0 = L.node_item0;
  a.node_nitems = L.node_nitems;
  a.n_items = (int)L.n_items;
  a.n_nodes = L.n_nodes;
  a.work = t->d_work;
  a.prefix = L.prefix;
  a.node_prob = L.prob;
  a.prob = t->d_prob;
  a.flags = L.flags;
  a.deg_used = L.deg_used;
  a.x = t->x;
  a.y = t->y;
  a.z = t->z;
  a.r = t->r;
  a.s = b.s;
  a.mstat = b.mstat;
  a.acc = b.acc;
  a.acc_stride = b.acc_stride;
  a.gacc = b.gacc;
  a.lcoef = b.lcoef;
  a.coef = L.coef;
  a.hcoef = L.hcoef;
  a.stride = t->nmono;
  a.depth = depth;
  a.MR = mrows_for(mixed_m_cap(L.max_m));
  a.tmem_cols = 32;
  a.nstages = 2;
  a.cache = b.cache;
  a.cache_mode = 0;
  a.cache_atom_bytes = 0;
  a.last_sweep = 0;
  a.err = t->d_err;
  a.tier = 1;
  a.rbuf = t->Rbuf;
  a.item_roff = L.item_roff;
  a.dproj = b.dproj;
  a.dstride = t->nmono;
  a.node_start = L.start;
  a.node_count = L.count;
  a.bd = level_bounds(t, depth);
  a.route_hard = route_hard(t, depth) ? 1 : 0;
  a.r_out = t->r;
  return a;
}

uint32_t pow2_cols(int c) {
  uint32_t v = 32;
  while ((int)v < c) v <<= 1;
  return v;
}

template <bool kProj>
cudaError_t launch_gram_t(const fmt_tree* t, int depth, const fmt_mixed_bufs& b, int cache_mode, cudaStream_t s) {
  const fmt_level& L = t->lv[depth];
  if (L.n_items <= 0) return cudaSuccess;
  MArgs a = make_margs(t, depth, b);
  a.cache_mode = b.cache ? cache_mode : 0;
  a.cache_atom_bytes = 4u * (uint32_t)a.MR * 128u;
  // projection: 4 digits x 2 bands x 16 columns; Gram: the two bands of the matrix
  a.tmem_cols = (int)pow2_cols(kProj ? 128 : gram_cols(mixed_m_cap(L.max_m)));
  const size_t stage = 4 * (size_t)a.MR * 128 + (kProj ? 2048 : 0);
  const size_t fixed = 1024 + kLegBytes + 12 * 1024;  // alignment, Legendre table, static shared
  a.nstages = fixed + 2 * stage <= 227 * 1024 ? 2 : 1;
  const size_t smem = 1024 + kLegBytes + a.nstages * stage;
  cudaError_t e = fmt_smem_at_least((const void*)k_mgram<kProj>, smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mgram<kProj>, kGThreads, smem)) != cudaSuccess)
    return e;
  if (per_sm < 1) per_sm = 1;
  const int tmem_cap = 512 / a.tmem_cols;  // tensor memory of an SM shared by its resident CTAs
  if (per_sm > tmem_cap) per_sm = tmem_cap;
  int64_t grid = (int64_t)nsm() * per_sm;
  if (grid > L.n_items) grid = L.n_items;
  if ((e = cudaMemsetAsync(t->d_work, 0, sizeof(int), s)) != cudaSuccess) return e;
  k_mgram<kProj><<<(unsigned)grid, kGThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

int mixed_m_cap(int max_m) {
  const int cap = fmt_nmono_d(FMT_MIXED_MAX_DEGREE) + 1;
  return max_m < cap ? max_m : cap;
}
size_t mixed_acc_stride(int max_m) { return (size_t)gram_cols(mixed_m_cap(max_m)) * 128; }

cudaError_t launch_mixed_box(const fmt_tree* t, int depth, const fmt_mixed_bufs& b, cudaStream_t s) {
  const fmt_level& L = t->lv[depth];
  if (L.n_items <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(b.mstat, 0, sizeof(unsigned long long) * kMStat * (size_t)L.n_nodes, s);
  if (e != cudaSuccess) return e;
  k_mbox<<<(unsigned)L.n_items, 256, 0, s>>>(make_margs(t, depth, b));
  return cudaGetLastError();
}

cudaError_t launch_mixed_gram(const fmt_tree* t, int depth, const fmt_mixed_bufs& b, bool projection,
                              int cache_mode, cudaStream_t s) {
  return projection ? launch_gram_t<true>(t, depth, b, cache_mode, s)
                    : launch_gram_t<false>(t, depth, b, cache_mode, s);
}

size_t mixed_cache_bytes(const fmt_tree* t, int depth) {
  const fmt_level& L = t->lv[depth];
  // atom index item + row/64 + atom < n_items + n/64 + 2
  return (size_t)(L.n_items + t->n / kAtom + 2) * 4 * (size_t)mrows_for(mixed_m_cap(L.max_m)) * 128;
}

size_t mixed_factor_smem(int max_m) {  // G | rk | invd | Fl; the conversion scratch reuses G, rk, invd
  return sizeof(double) * ((size_t)ro_of(max_m, max_m) + 3 * (size_t)max_m);
}

cudaError_t launch_mixed_factor(const fmt_tree* t, int depth, const fmt_mixed_bufs& b, cudaStream_t s) {
  const fmt_level& L = t->lv[depth];
  if (L.n_nodes <= 0) return cudaSuccess;
  {
    const int chunks = (int)((mixed_acc_stride(L.max_m) + kRedChunk - 1) / kRedChunk);
    k_mreduce<<<(unsigned)(L.n_nodes * chunks), 256, 0, s>>>(make_margs(t, depth, b), chunks);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const size_t smem = mixed_factor_smem(mixed_m_cap(L.max_m));
  cudaError_t e = cudaMemsetAsync(t->d_work + kPivSlot, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  e = fmt_smem_at_least((const void*)k_mfactor, smem);
  if (e != cudaSuccess) return e;
  k_mfactor<<<(unsigned)L.n_nodes, kFThreads, smem, s>>>(make_margs(t, depth, b));
  return cudaGetLastError();
}

cudaError_t launch_mixed_sresid(const fmt_tree* t, int depth, const fmt_mixed_bufs& b, cudaStream_t s) {
  const fmt_level& L = t->lv[depth];
  if (L.n_items <= 0) return cudaSuccess;
  k_msresid<true><<<(unsigned)L.n_items, 256, 0, s>>>(make_margs(t, depth, b));
  return cudaGetLastError();
}

cudaError_t launch_mixed_final_residual(const fmt_tree* t, int depth, const fmt_mixed_bufs& b, cudaStream_t s) {
  const fmt_level& L = t->lv[depth];
  if (L.n_items <= 0) return cudaSuccess;
  MArgs a = make_margs(t, depth, b);
  k_mresid_final<<<(unsigned)L.n_items, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_mixed_update(const fmt_tree* t, int depth, const fmt_mixed_bufs& b, bool last,
                                cudaStream_t s) {
  const fmt_level& L = t->lv[depth];
  if (L.n_nodes <= 0) return cudaSuccess;
  MArgs a = make_margs(t, depth, b);
  a.last_sweep = last ? 1 : 0;
  const int mc = mixed_m_cap(L.max_m);
  const size_t smem = sizeof(double) * ((size_t)ro_of(mc, mc) + 3 * (size_t)mc);
  cudaError_t e = fmt_smem_at_least((const void*)k_mupdate, smem);
  if (e != cudaSuccess) return e;
  k_mupdate<<<(unsigned)L.n_nodes, kFThreads, smem, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- tier 2 launchers
size_t tier2_factor_smem(int max_m) {
  return sizeof(double) * ((size_t)(kPanel + kRT + 3) * max_m + conv_ws_doubles(FMT_MAX_DEGREE));
}

cudaError_t launch_tier2_gram(const fmt_tree* t, int depth, const fmt_mixed_bufs& b, cudaStream_t s) {
  const fmt_level& L = t->lv[depth];
  if (L.n_items <= 0) return cudaSuccess;
  const int nt = (L.max_m + kDT - 1) / kDT, npairs = nt * (nt + 1) / 2;
  k_dgram<<<(unsigned)(L.n_items * npairs), 256, 0, s>>>(make_margs(t, depth, b), npairs);
  return cudaGetLastError();
}

cudaError_t launch_tier2_factor(const fmt_tree* t, int depth, const fmt_mixed_bufs& b, cudaStream_t s) {
  const fmt_level& L = t->lv[depth];
  if (L.n_nodes <= 0) return cudaSuccess;
  const size_t smem = tier2_factor_smem(L.max_m);
  cudaError_t e = fmt_smem_at_least((const void*)k_dfactor, smem);
  if (e != cudaSuccess) return e;
  k_dfactor<<<(unsigned)L.n_nodes, 256, smem, s>>>(make_margs(t, depth, b));
  return cudaGetLastError();
}

cudaError_t launch_tier2_sweep(const fmt_tree* t, int depth, const fmt_mixed_bufs& b, int part, bool last,
                               cudaStream_t s) {
  const fmt_level& L = t->lv[depth];
  if (L.n_items <= 0) return cudaSuccess;
  MArgs a = make_margs(t, depth, b);
  a.tier = 2;
  a.last_sweep = last ? 1 : 0;
  if (part == 0) {
    k_msresid<false><<<(unsigned)L.n_items, 256, 0, s>>>(a);
  } else if (part == 1) {
    k_dproj<<<(unsigned)L.n_items, 256, 0, s>>>(a);
  } else {
    const size_t smem = sizeof(double) * (3 * (size_t)L.max_m + conv_ws_doubles(FMT_MAX_DEGREE));
    cudaError_t e = fmt_smem_at_least((const void*)k_dupdate, smem);
    if (e != cudaSuccess) return e;
    k_dupdate<<<(unsigned)L.n_nodes, kFThreads, smem, s>>>(a);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- bounded-wait probe
namespace {
// One thread waits on an mbarrier that nothing arrives on, through the same
// bounded wait as the kernels above; when the bound runs out it records
// FMT_ERR_TIMEOUT in the error word and returns (no trap, no hang).
__global__ void k_wait_probe(unsigned long long limit_ns, int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_mbar_init();
  if (!mbar_wait_for(&bar, 0, limit_ns)) atomicOr(err, FMT_ERR_TIMEOUT);
}
}  // namespace

cudaError_t launch_wait_probe(unsigned long long limit_ns, int* d_err, cudaStream_t s) {
  k_wait_probe<<<1, 32, 0, s>>>(limit_ns, d_err);
  return cudaGetLastError();
}

#ifdef FMT_CHECKED
FMT_CHECK_READER(check_site_mixed)
#endif
