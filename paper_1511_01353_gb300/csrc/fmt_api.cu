// fmt_api.cu -- the C ABI of libfmt (declared in include/fmt.h): argument
// checks, the tree's memory (a stream-ordered pool per device), the
// call-order state machine, and the sequence of kernels behind oct_build /
// oct_build_batch / fit_level / refine / evaluate (FP64 path; the mixed
// path's tensor-core tier, its FP64 normal-equations tier and the Householder
// refits in one level step).  Also here: the CUDA-graph form of fit_level
// (one executable graph per level step, updated in place), the versioned
// export / import of a tree (the import checks the whole host blob before
// any device work), kernel profiling by CUDA events, and the failure-path
// diagnostics (allocation-failure injection, the bounded-wait probe).
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <new>

#include "fmt_internal.cuh"

namespace {

thread_local char g_msg[256] = "no error";

fmt_status set_err(fmt_tree* t, fmt_status st, const char* fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (t) {
    memcpy(t->msg, buf, sizeof(buf));
    if (st == FMT_ECUDA || st == FMT_EINTERNAL) t->sticky = st;
  }
  memcpy(g_msg, buf, sizeof(buf));
  return st;
}

std::mutex g_mu;
cudaMemPool_t g_pool[64];
bool g_inited[64];

fmt_status device_init(int dev) {
  if (dev < 0 || dev >= 64) return set_err(nullptr, FMT_ECUDA, "device id %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_inited[dev]) return FMT_OK;
  cudaMemPoolProps props;
  memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaError_t e = cudaMemPoolCreate(&g_pool[dev], &props);
  if (e != cudaSuccess) return set_err(nullptr, FMT_ECUDA, "memory pool: %s", cudaGetErrorString(e));
  uint64_t thr = UINT64_MAX;  // keep freed blocks cached in the pool
  cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &thr);
  g_inited[dev] = true;
  return FMT_OK;
}

// ---------------------------------------------------------------- profiling
enum {
  K_CHECK = 0, K_MORTON, K_SORT, K_GATHER, K_PLAN, K_TILE_QR, K_COMBINE, K_BACKSOLVE,
  K_RESIDUAL, K_CHILD, K_REFINE, K_EVALUATE, K_HCOEF, K_MBOX, K_MGRAM, K_MFACTOR, K_MSRESID, K_MPROJ,
  K_MUPDATE, K_GRAPH, K_DGRAM, K_DFACTOR, K_DPROJ, K_DUPDATE, K_NCLASS
};
static_assert(K_NCLASS <= FMT_PROFILE_CLASSES, "profile classes exceed FMT_PROFILE_CLASSES");
const char* const kClassNames[K_NCLASS] = {"check_maxabs", "morton", "radix_sort", "gather", "plan_root",
                                           "tile_qr", "combine", "back_solve", "residual", "child_stats",
                                           "refine", "evaluate", "make_hcoef", "mixed_box", "mixed_gram",
                                           "mixed_factor", "mixed_sresid", "mixed_proj", "mixed_update",
                                           "graph_launch", "fp64_gram", "fp64_factor", "fp64_proj",
                                           "fp64_update"};
struct ProfRec {
  int k;
  cudaEvent_t a, b;
};
std::mutex g_pmu;
bool g_prof_on = false;
int64_t g_launch[FMT_PROFILE_CLASSES];
double g_units[FMT_PROFILE_CLASSES];
double g_flops[FMT_PROFILE_CLASSES];
ProfRec* g_recs = nullptr;
int64_t g_nrecs = 0, g_caprecs = 0;
cudaEvent_t* g_evpool = nullptr;
int64_t g_nev = 0;

cudaEvent_t prof_event() {
  if (g_nev > 0) return g_evpool[--g_nev];
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Counts the launches of one kernel class and, while profiling is on, brackets
// them with events on the launching stream.
struct ProfScope {
  int k;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  bool on = false;
  ProfScope(int k_, cudaStream_t s_, int nlaunch, double units, double flops) : k(k_), s(s_) {
    std::lock_guard<std::mutex> lk(g_pmu);
    g_launch[k] += nlaunch;
    g_units[k] += units;
    g_flops[k] += flops;
    if (g_prof_on) {
      a = prof_event();
      if (a && record(a) == cudaSuccess) on = true;
    }
  }
  // Inside a stream capture the events become event-record nodes of the
  // graph (recorded at every replay), so timing works in both modes.
  cudaError_t record(cudaEvent_t ev) const {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
      return cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
    return cudaEventRecord(ev, s);
  }
  ~ProfScope() {
    if (!on) return;
    std::lock_guard<std::mutex> lk(g_pmu);
    cudaEvent_t b = prof_event();
    if (!b || record(b) != cudaSuccess) return;
    if (g_nrecs == g_caprecs) {
      int64_t nc = g_caprecs ? 2 * g_caprecs : 1024;
      ProfRec* nr = (ProfRec*)realloc(g_recs, sizeof(ProfRec) * (size_t)nc);
      if (!nr) return;
      g_recs = nr;
      g_caprecs = nc;
    }
    g_recs[g_nrecs++] = ProfRec{k, a, b};
  }
};

// fmt_debug_fail_alloc: > 0 counts down the device allocations; the one that
// takes it from 1 to 0 fails as if the device were out of memory
std::atomic<int64_t> g_fail_alloc{0};

template <typename T>
fmt_status talloc(fmt_tree* t, T** p, int64_t count, cudaStream_t s) {
  size_t bytes = (size_t)(count > 0 ? count : 1) * sizeof(T);
  bytes = (bytes + 255) & ~(size_t)255;
  for (int64_t k = g_fail_alloc.load(); k > 0; k = g_fail_alloc.load())
    if (g_fail_alloc.compare_exchange_weak(k, k - 1)) {
      if (k == 1) return set_err(t, FMT_ENOMEM, "device allocation of %zu bytes failed (injected)", bytes);
      break;
    }
  void* ptr = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&ptr, bytes, g_pool[t->device], s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(t, FMT_ENOMEM, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  if (t->n_allocs == t->cap_allocs) {
    int nc = t->cap_allocs ? 2 * t->cap_allocs : 64;
    void** na = (void**)realloc(t->allocs, sizeof(void*) * (size_t)nc);
    if (!na) {
      cudaFreeAsync(ptr, s);
      return set_err(t, FMT_ENOMEM, "host allocation failed");
    }
    t->allocs = na;
    t->cap_allocs = nc;
  }
  t->allocs[t->n_allocs++] = ptr;
  *p = (T*)ptr;
  return FMT_OK;
}

void tfree_one(fmt_tree* t, void* ptr, cudaStream_t s) {
  for (int i = 0; i < t->n_allocs; ++i)
    if (t->allocs[i] == ptr) {
      cudaFreeAsync(ptr, s);
      t->allocs[i] = t->allocs[--t->n_allocs];
      return;
    }
}

#define TRY(expr)                 \
  do {                            \
    fmt_status st_ = (expr);      \
    if (st_ != FMT_OK) return st_; \
  } while (0)

#define CUDA_TRY(t, expr, what)                                                         \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess) return set_err(t, FMT_ECUDA, "%s: %s", what, cudaGetErrorString(e_)); \
  } while (0)

int64_t nmin_of(const fmt_tree* t) {
  // the smallest child any problem of the forest can create
  int64_t v = t->P.min_pts > fmt_nmono(0) ? t->P.min_pts : 1;
  int32_t dmin = t->max_degree;
  for (int64_t i = 0; i < t->n_problems; ++i)
    if (t->h_prob[i].degree < dmin) dmin = t->h_prob[i].degree;
  if (fmt_nmono(dmin) > v) v = fmt_nmono(dmin);
  return v < 1 ? 1 : v;
}

int64_t min_chunk(const fmt_tree* t) {
  return t->P.chunk_rows > 0 ? t->P.chunk_rows : t->chunk_floor;
}

fmt_status alloc_level(fmt_tree* t, int d, int64_t cap_nodes, int64_t cap_items, cudaStream_t s) {
  fmt_level& L = t->lv[d];
  L.cap_nodes = cap_nodes;
  L.cap_items = cap_items;
  const int64_t nm = t->nmono;
  TRY(talloc(t, &L.prefix, cap_nodes, s));
  TRY(talloc(t, &L.prob, cap_nodes, s));
  TRY(talloc(t, &L.start, cap_nodes, s));
  TRY(talloc(t, &L.count, cap_nodes, s));
  TRY(talloc(t, &L.flags, cap_nodes, s));
  TRY(talloc(t, &L.deg_used, cap_nodes, s));
  TRY(talloc(t, &L.masks, cap_nodes, s));
  TRY(talloc(t, &L.bounds, 9 * cap_nodes, s));
  TRY(talloc(t, &L.child_S, 8 * cap_nodes, s));
  TRY(talloc(t, &L.child_n, 8 * cap_nodes, s));
  TRY(talloc(t, &L.child_E, 8 * cap_nodes, s));
  TRY(talloc(t, &L.coef, nm * cap_nodes, s));
  TRY(talloc(t, &L.hcoef, nm * cap_nodes, s));
  TRY(talloc(t, &L.ccoef, nm * cap_nodes, s));
  TRY(talloc(t, &L.frame, 6 * cap_nodes, s));
  if (t->P.precision == FMT_MIXED) TRY(talloc(t, &L.ccoef_df, ((nm + 1) & ~1) * cap_nodes, s));  // fmt_horner_df
  TRY(talloc(t, &L.node_item0, cap_nodes, s));
  TRY(talloc(t, &L.node_nitems, cap_nodes, s));
  TRY(talloc(t, &L.item_node, cap_items, s));
  TRY(talloc(t, &L.item_start, cap_items, s));
  TRY(talloc(t, &L.item_end, cap_items, s));
  TRY(talloc(t, &L.item_local, cap_items, s));
  TRY(talloc(t, &L.sched, cap_items, s));
  TRY(talloc(t, &L.item_roff, cap_items, s));
  CUDA_TRY(t, cudaMemsetAsync(L.masks, 0, sizeof(int32_t) * (size_t)cap_nodes, s), "memset");
  CUDA_TRY(t, cudaMemsetAsync(L.child_E, 0, sizeof(double) * 8 * (size_t)cap_nodes, s), "memset");
  return FMT_OK;
}

fmt_status check_tree(fmt_tree* t) {
  if (!t) return set_err(nullptr, FMT_EINVAL, "tree is NULL");
  if (t->sticky != FMT_OK) return t->sticky;
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != t->device)
    return set_err(t, FMT_EINVAL, "current device %d differs from the tree's device %d", dev, t->device);
  return FMT_OK;
}

// read back the plan block and the device error word
fmt_status read_plan(fmt_tree* t, cudaStream_t s) {
  CUDA_TRY(t, cudaMemcpyAsync(t->h_plan, t->d_plan, sizeof(fmt_plan_out), cudaMemcpyDeviceToHost, s), "plan copy");
  CUDA_TRY(t, cudaMemcpyAsync(t->h_err, t->d_err, sizeof(int), cudaMemcpyDeviceToHost, s), "err copy");
  CUDA_TRY(t, cudaStreamSynchronize(s), "synchronise");
  t->h_plan->err = *t->h_err;
  return FMT_OK;
}

void destroy(fmt_tree* t) {
  if (!t) return;
  cudaDeviceSynchronize();
  for (int i = 0; i < t->n_allocs; ++i) cudaFreeAsync(t->allocs[i], 0);
  cudaStreamSynchronize(0);
  for (int q = 0; q <= FMT_MAX_DEGREE; ++q) {
    if (t->side[q]) cudaStreamDestroy(t->side[q]);
    if (t->join_ev[q]) cudaEventDestroy(t->join_ev[q]);
  }
  if (t->fork_ev) cudaEventDestroy(t->fork_ev);
  if (t->piv_stream) cudaStreamDestroy(t->piv_stream);
  if (t->piv_fork) cudaEventDestroy(t->piv_fork);
  if (t->piv_join) cudaEventDestroy(t->piv_join);
  free(t->allocs);
  if (t->h_plan) cudaFreeHost(t->h_plan);
  if (t->h_err) cudaFreeHost(t->h_err);
  free(t->h_prob);
  delete t;
}

int bits_for(int64_t v) {  // bits to hold the values 0 .. v-1
  int b = 0;
  while (b < 62 && (int64_t(1) << b) < v) ++b;
  return b;
}

fmt_status validate_shared(const fmt_params& P) {
  if (P.max_depth < 0 || P.max_depth > FMT_MAX_DEPTH)
    return set_err(nullptr, FMT_EINVAL, "max_depth %d outside [0, %d]", P.max_depth, FMT_MAX_DEPTH);
  if (P.min_pts < 0) return set_err(nullptr, FMT_EINVAL, "min_pts %d < 0", P.min_pts);
  if (P.precision != FMT_FP64 && P.precision != FMT_MIXED)
    return set_err(nullptr, FMT_EINVAL, "precision must be FMT_FP64 or FMT_MIXED");
  if (P.sweeps < -1 || P.sweeps > FMT_MIXED_MAX_SWEEPS)
    return set_err(nullptr, FMT_EINVAL, "sweeps %d outside [-1, %d]", P.sweeps, FMT_MIXED_MAX_SWEEPS);
  if ((P.options & ~FMT_OPT_GRAPH) != 0) return set_err(nullptr, FMT_EINVAL, "options has unknown bits (0x%x)", P.options);
  if (!(P.tol_rel >= 0.0) || !isfinite(P.tol_rel)) return set_err(nullptr, FMT_EINVAL, "tol_rel must be finite, >= 0");
  if (P.chunk_rows < 0) return set_err(nullptr, FMT_EINVAL, "chunk_rows < 0");
  return FMT_OK;
}

fmt_status validate_box(double lo0, double lo1, double lo2, double side) {
  if (!(side > 0.0) || !isfinite(side)) return set_err(nullptr, FMT_EINVAL, "side must be finite, > 0");
  if (!isfinite(lo0) || !isfinite(lo1) || !isfinite(lo2)) return set_err(nullptr, FMT_EINVAL, "lo must be finite");
  return FMT_OK;
}

// Stage a forest of n_problems independent problems (offsets[p] .. offsets[p+1]
// of the inputs) and build its roots.
fmt_status build_forest(const fmt_params* params, int64_t P, const int64_t* offsets, const int32_t* degrees,
                        const double* boxes, const double* x, const double* y, const double* z, const double* f,
                        cudaStream_t s, fmt_tree** out) {
  if (!out) return set_err(nullptr, FMT_EINVAL, "out is NULL");
  *out = nullptr;
  if (!params) return set_err(nullptr, FMT_EINVAL, "params is NULL");
  const fmt_params& PP = *params;
  TRY(validate_shared(PP));
  if (P < 1) return set_err(nullptr, FMT_EINVAL, "n_problems = %lld < 1", (long long)P);
  if (!offsets || offsets[0] != 0) return set_err(nullptr, FMT_EINVAL, "offsets must start at 0");
  for (int64_t i = 0; i < P; ++i)
    if (offsets[i + 1] <= offsets[i])
      return set_err(nullptr, FMT_EINVAL, "problem %lld has no point (offsets must increase)", (long long)i);
  const int64_t n = offsets[P];
  if (n > (int64_t)0xfffffffe) return set_err(nullptr, FMT_EINVAL, "n = %lld above 2^32-2 points", (long long)n);
  if (!x || !y || !z || !f) return set_err(nullptr, FMT_EINVAL, "NULL input pointer");
  int32_t maxdeg = -1, mindeg = FMT_MAX_DEGREE + 1;
  for (int64_t i = 0; i < P; ++i) {
    const int32_t p = degrees ? degrees[i] : PP.degree;
    if (p < 0 || p > FMT_MAX_DEGREE)
      return set_err(nullptr, FMT_EINVAL, "degree %d outside [0, %d]", p, FMT_MAX_DEGREE);
    if (p > maxdeg) maxdeg = p;
    if (p < mindeg) mindeg = p;
    const double* b = boxes ? boxes + 4 * i : nullptr;
    TRY(validate_box(b ? b[0] : PP.lo[0], b ? b[1] : PP.lo[1], b ? b[2] : PP.lo[2], b ? b[3] : PP.side));
  }
  const int sort_levels = PP.max_depth + 1 < FMT_QBITS ? PP.max_depth + 1 : FMT_QBITS;
  const int sort_bits = 3 * sort_levels;
  const int pid_bits = P > 1 ? bits_for(P) : 0;
  if (pid_bits + sort_bits > 64 || pid_bits + 3 * PP.max_depth > 63)
    return set_err(nullptr, FMT_EINVAL, "%lld problems need %d key bits: lower max_depth (at most %d here)",
                   (long long)P, pid_bits, (63 - pid_bits) / 3 - 1);
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return set_err(nullptr, FMT_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(ce));
  TRY(device_init(dev));

  fmt_tree* t = new (std::nothrow) fmt_tree();
  if (!t) return set_err(nullptr, FMT_ENOMEM, "host allocation failed");
  auto fail = [&](fmt_status e) {
    destroy(t);
    return e;
  };
  t->P = PP;
  if (t->P.chunk_rows > 0) t->P.chunk_rows = (t->P.chunk_rows + 63) / 64 * 64;
  t->device = dev;
  t->stream = s;
  t->n = n;
  t->n_problems = P;
  t->max_degree = maxdeg;
  t->nmono = fmt_nmono(maxdeg);
  t->sort_bits = sort_bits;
  t->pid_bits = pid_bits;
  {
    // A chunk of C rows costs about 2 m^2 C flops and one merge about (2/3) m^3,
    // so C >= 4m keeps merges under ~10% of the chunk work (the built-in
    // factor 4; the autotuner may pick another, which a tree of one degree
    // uses: the floor is tree-wide, and a tuned factor measured on one degree
    // does not carry over to a forest's mix); above that floor the planner
    // sizes chunks to the rows per resident QR CTA, so that the largest item
    // is no longer than the average share of a CTA.
    const int64_t factor = mindeg == maxdeg ? qr_config(t->nmono + 1).chunk_factor : 4;
    int64_t fl = factor * (int64_t)(t->nmono + 1);
    t->chunk_floor = fl < 64 ? 64 : (fl + 63) / 64 * 64;
  }
  t->h_prob = (fmt_problem*)calloc((size_t)P, sizeof(fmt_problem));
  if (!t->h_prob) {
    set_err(nullptr, FMT_ENOMEM, "host allocation failed");
    return fail(FMT_ENOMEM);
  }
  for (int64_t i = 0; i < P; ++i) {
    fmt_problem& pr = t->h_prob[i];
    const double* b = boxes ? boxes + 4 * i : nullptr;
    pr.lo[0] = b ? b[0] : PP.lo[0];
    pr.lo[1] = b ? b[1] : PP.lo[1];
    pr.lo[2] = b ? b[2] : PP.lo[2];
    pr.side = b ? b[3] : PP.side;
    pr.S = 2097152.0 / pr.side;
    pr.inv_side = 1.0 / pr.side;
    for (int a = 0; a < 3; ++a) pr.hi[a] = pr.lo[a] + pr.side;
    pr.degree = degrees ? degrees[i] : PP.degree;
    pr.start = offsets[i];
    pr.count = offsets[i + 1] - offsets[i];
    int32_t q = pr.degree;
    if (pr.count < fmt_nmono(q)) {
      q = -1;
      while (fmt_nmono(q + 1) <= pr.count) ++q;
    }
    pr.q_root = q;
  }
  if (P == 1) {  // the single-problem parameters mirror problem 0
    t->P.degree = t->h_prob[0].degree;
    t->P.lo[0] = t->h_prob[0].lo[0];
    t->P.lo[1] = t->h_prob[0].lo[1];
    t->P.lo[2] = t->h_prob[0].lo[2];
    t->P.side = t->h_prob[0].side;
  }
  const bool key64 = pid_bits + sort_bits > 32;
  const int sort_shift = 3 * (FMT_QBITS - sort_levels);

  fmt_status st = FMT_OK;
  void *keys = nullptr, *keys_alt = nullptr, *temp = nullptr;
  uint32_t *vals = nullptr, *vals_alt = nullptr;
  unsigned long long* d_maxbits = nullptr;
  const size_t ksz = key64 ? 8 : 4;
  if ((st = talloc(t, &t->x, n, s)) || (st = talloc(t, &t->y, n, s)) || (st = talloc(t, &t->z, n, s)) ||
      (st = talloc(t, &t->r, n, s)) || (st = talloc(t, &t->code, n, s)) ||
      (st = talloc(t, (char**)&keys, (int64_t)ksz * n, s)) || (st = talloc(t, (char**)&keys_alt, (int64_t)ksz * n, s)) ||
      (st = talloc(t, &vals, n, s)) || (st = talloc(t, &vals_alt, n, s)) ||
      (st = talloc(t, (char**)&temp, (int64_t)radix_sort_temp_bytes(n, key64), s)) ||
      (st = talloc(t, &t->d_err, 1, s)) || (st = talloc(t, &d_maxbits, P, s)) ||
      (st = talloc(t, &t->d_plan, 1, s)) || (st = talloc(t, &t->d_counter, 1, s)) ||
      (st = talloc(t, &t->d_work, kWorkSlots, s)) || (st = talloc(t, &t->d_prob, P, s)))
    return fail(st);
  if (cudaMallocHost((void**)&t->h_plan, sizeof(fmt_plan_out)) != cudaSuccess ||
      cudaMallocHost((void**)&t->h_err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    set_err(nullptr, FMT_ENOMEM, "pinned host allocation failed");
    return fail(FMT_ENOMEM);
  }
  // roots: one node per problem
  const int64_t cap_items0 = n / min_chunk(t) + P + 2;
  if ((st = alloc_level(t, 0, P, cap_items0, s))) return fail(st);

  cudaError_t e = cudaSuccess;
  void* kout = nullptr;
  uint32_t* vout = nullptr;
  do {
    if ((e = cudaMemcpyAsync(t->d_prob, t->h_prob, sizeof(fmt_problem) * (size_t)P, cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
      break;
    if ((e = cudaMemsetAsync(t->d_err, 0, sizeof(int), s)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(d_maxbits, 0, sizeof(unsigned long long) * (size_t)P, s)) != cudaSuccess) break;
    {
      ProfScope ps(K_CHECK, s, 1, (double)n, 0.0);
      if ((e = launch_check_maxabs(n, x, y, z, f, t->d_prob, (int)P, d_maxbits, t->d_err, s)) != cudaSuccess) break;
    }
    {
      ProfScope ps(K_MORTON, s, 1, (double)n, 0.0);
      e = launch_morton(n, x, y, z, t->d_prob, (int)P, sort_shift, sort_bits, key64, keys, vals, s);
      if (e != cudaSuccess) break;
    }
    {
      const int bits = pid_bits + sort_bits;
      ProfScope ps(K_SORT, s, 4 * ((bits + 7) / 8), (double)n, 0.0);
      e = launch_radix_sort(n, bits, key64, keys, vals, keys_alt, vals_alt, temp, &kout, &vout, s);
      if (e != cudaSuccess) break;
    }
    t->perm = vout;
    {
      ProfScope ps(K_GATHER, s, 1, (double)n, 0.0);
      e = launch_gather(n, t->perm, x, y, z, f, t->d_prob, (int)P, t->x, t->y, t->z, t->r, t->code, s);
    }
  } while (0);
  if (e != cudaSuccess) {
    set_err(nullptr, FMT_ECUDA, "oct_build launch: %s", cudaGetErrorString(e));
    return fail(FMT_ECUDA);
  }
  // per-problem tau = tol_rel * max |f| (host), then the roots
  unsigned long long* hbits = (unsigned long long*)malloc(sizeof(unsigned long long) * (size_t)P);
  if (!hbits) {
    set_err(nullptr, FMT_ENOMEM, "host allocation failed");
    return fail(FMT_ENOMEM);
  }
  if ((e = cudaMemcpyAsync(hbits, d_maxbits, sizeof(unsigned long long) * (size_t)P, cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(t->h_err, t->d_err, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    free(hbits);
    set_err(nullptr, FMT_ECUDA, "copy: %s", cudaGetErrorString(e));
    return fail(FMT_ECUDA);
  }
  if (*t->h_err & FMT_ERR_NONFINITE) {
    free(hbits);
    set_err(nullptr, FMT_EINVAL, "non-finite coordinate or value in the input");
    return fail(FMT_EINVAL);
  }
  for (int64_t i = 0; i < P; ++i) {
    double mx;
    memcpy(&mx, &hbits[i], sizeof(mx));
    t->h_prob[i].maxabs = mx;
    t->h_prob[i].tau = PP.tol_rel * mx;
  }
  free(hbits);
  t->maxabs = t->h_prob[0].maxabs;
  t->tau = t->h_prob[0].tau;
  if ((e = cudaMemcpyAsync(t->d_prob, t->h_prob, sizeof(fmt_problem) * (size_t)P, cudaMemcpyHostToDevice, s)) !=
      cudaSuccess) {
    set_err(nullptr, FMT_ECUDA, "copy: %s", cudaGetErrorString(e));
    return fail(FMT_ECUDA);
  }
  {
    ProfScope ps(K_PLAN, s, 1, (double)P, 0.0);
    e = launch_plan_root(t, t->P.chunk_rows, t->chunk_floor, t->d_plan, s);
  }
  if (e != cudaSuccess) {
    set_err(nullptr, FMT_ECUDA, "oct_build launch: %s", cudaGetErrorString(e));
    return fail(FMT_ECUDA);
  }
  if (read_plan(t, s) != FMT_OK) {
    set_err(nullptr, FMT_ECUDA, "%s", t->msg);
    return fail(FMT_ECUDA);
  }
  const fmt_plan_out& pl = *t->h_plan;
  if (pl.err) {
    set_err(nullptr, FMT_EINTERNAL, "device check failed in oct_build (0x%llx)", (unsigned long long)pl.err);
    return fail(FMT_EINTERNAL);
  }
  fmt_level& L0 = t->lv[0];
  L0.n_nodes = P;
  L0.n_items = pl.n_items;
  L0.max_chunks = pl.max_chunks;
  L0.chunk_rows = pl.chunk_rows;
  L0.n_points = n;
  L0.max_m = (int32_t)pl.max_m;
  L0.deg_mask = pl.deg_mask;
  L0.r_total = pl.r_total;
  L0.n_hard_items = pl.n_hard_items;
  L0.qr_flops = pl.qr_flops;
  L0.horner_flops = pl.horner_flops;
  t->n_levels = 1;
  t->next_fit = 0;
  t->next_refine = -1;
  // the sort buffers are not needed any more (the permutation stays)
  tfree_one(t, keys, s);
  tfree_one(t, keys_alt, s);
  tfree_one(t, temp, s);
  tfree_one(t, vout == vals ? (void*)vals_alt : (void*)vals, s);
  tfree_one(t, d_maxbits, s);
  if (check_end(t, s) != FMT_OK) {
    set_err(nullptr, FMT_EINTERNAL, "%s", t->msg);
    return fail(FMT_EINTERNAL);
  }
  *out = t;
  return FMT_OK;
}

// Grows the mixed path's scratch to the level's needs.
fmt_status ensure_mixed(fmt_tree* t, int depth, cudaStream_t s) {
  const fmt_level& L = t->lv[depth];
  fmt_mixed_bufs& b = t->mx;
  if (!b.s) TRY(talloc(t, &b.s, t->n, s));
  if (b.cap_nodes < L.n_nodes) {
    if (b.mstat) tfree_one(t, b.mstat, s);
    if (b.lcoef) tfree_one(t, b.lcoef, s);
    b.mstat = nullptr;
    b.lcoef = nullptr;
    b.cap_nodes = 0;
    TRY(talloc(t, &b.mstat, 8 * L.n_nodes, s));
    TRY(talloc(t, &b.lcoef, (int64_t)t->nmono * L.n_nodes, s));
    b.cap_nodes = L.n_nodes;
  }
  if (b.cap_items < L.n_items) {
    if (b.gacc) tfree_one(t, b.gacc, s);
    b.gacc = nullptr;
    b.cap_items = 0;
    TRY(talloc(t, &b.gacc, 256 * L.n_items, s));
    b.cap_items = L.n_items;
  }
  if (b.cap_dproj < L.n_items * (int64_t)t->nmono) {
    if (b.dproj) tfree_one(t, b.dproj, s);
    b.dproj = nullptr;
    b.cap_dproj = 0;
    TRY(talloc(t, &b.dproj, L.n_items * (int64_t)t->nmono, s));
    b.cap_dproj = L.n_items * (int64_t)t->nmono;
  }
  // basis cache of the sweeps, unless it would exceed kCacheCap (then each sweep regenerates)
  const size_t cache = mixed_cache_bytes(t, depth);
  constexpr size_t kCacheCap = (size_t)16 << 30;
  if (cache <= kCacheCap && b.cap_cache < cache) {
    if (b.cache) tfree_one(t, b.cache, s);
    b.cache = nullptr;
    b.cap_cache = 0;
    if (talloc(t, &b.cache, (int64_t)cache, s) == FMT_OK) b.cap_cache = cache;
  }
  b.acc_stride = (int64_t)mixed_acc_stride(L.max_m);
  const int64_t need = b.acc_stride * L.n_items;
  if (b.cap_acc < need) {
    if (b.acc) tfree_one(t, b.acc, s);
    b.acc = nullptr;
    b.cap_acc = 0;
    TRY(talloc(t, &b.acc, need, s));
    b.cap_acc = need;
  }
  return FMT_OK;
}

// The mixed-precision fit of one level (fmt_mixed.cu): nodes it fits carry
// FMT_FLAG_MIXED afterwards and are skipped by the FP64 kernels.
fmt_status fit_level_mixed(fmt_tree* t, int depth, cudaStream_t s) {
  const fmt_level& L = t->lv[depth];
  fmt_mixed_bufs b = t->mx;
  if (b.cap_cache < mixed_cache_bytes(t, depth)) b.cache = nullptr;  // too large: regenerate per sweep
  const double rows = (double)L.n_points, nodes = (double)L.n_nodes;
  // Householder refits beside the tensor-core tier run on a side stream; the
  // nearly square nodes (fewer than 1.5 m points), which the normal-equations
  // tiers often cannot fit, start there right away when the level has few
  // (route_hard).  Their QR scratch
  // slots are not used by the FP64 tier, which skips them.
  {
    cudaError_t e = cudaSuccess;
    if (!t->piv_stream) e = cudaStreamCreateWithFlags(&t->piv_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && !t->piv_fork) e = cudaEventCreateWithFlags(&t->piv_fork, cudaEventDisableTiming);
    if (e == cudaSuccess && !t->piv_join) e = cudaEventCreateWithFlags(&t->piv_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(t->piv_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(t->piv_stream, t->piv_fork, 0);
    if (e == cudaSuccess && route_hard(t, depth)) {
      ProfScope ps(K_TILE_QR, t->piv_stream, 1, 0.0, 0.0);
      e = launch_tile_qr(t, depth, t->Rbuf, t->piv_stream, 3);
    }
    CUDA_TRY(t, e, "nearly square nodes: Householder launch");
  }
  {
    ProfScope ps(K_MBOX, s, 2, rows, 0.0);
    CUDA_TRY(t, launch_mixed_box(t, depth, b, s), "mixed box launch");
  }
  {
    ProfScope ps(K_MGRAM, s, 1, rows, 0.0);
    CUDA_TRY(t, launch_mixed_gram(t, depth, b, false, 1, s), "mixed Gram launch");
  }
  {
    ProfScope ps(K_MFACTOR, s, 1, nodes, 0.0);
    CUDA_TRY(t, launch_mixed_factor(t, depth, b, s), "mixed factor launch");
  }
  // Nodes whose Cholesky pivot was too small go to Householder: refit them on
  // the side stream (after the nearly square ones) while the sweeps run;
  // fit_level_launches joins it before the other Householder refits.
  {
    cudaError_t e = cudaEventRecord(t->piv_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(t->piv_stream, t->piv_fork, 0);
    if (e == cudaSuccess) {
      ProfScope ps(K_TILE_QR, t->piv_stream, 1, 0.0, 0.0);
      e = launch_tile_qr(t, depth, t->Rbuf, t->piv_stream, 1);
    }
    if (e == cudaSuccess) e = cudaEventRecord(t->piv_join, t->piv_stream);
    CUDA_TRY(t, e, "early Householder refit launch");
    t->piv_pending = true;
  }
  const int sweeps = t->P.sweeps == 0 ? FMT_MIXED_MAX_SWEEPS : (t->P.sweeps < 0 ? 0 : t->P.sweeps);
  for (int k = 0; k < sweeps; ++k) {
    {
      ProfScope ps(K_MSRESID, s, 1, rows, L.horner_flops);
      CUDA_TRY(t, launch_mixed_sresid(t, depth, b, s), "mixed sweep residual launch");
    }
    {
      ProfScope ps(K_MPROJ, s, 1, rows, 0.0);
      CUDA_TRY(t, launch_mixed_gram(t, depth, b, true, 2, s), "mixed projection launch");
    }
    {
      ProfScope ps(K_MUPDATE, s, 1, nodes, 0.0);
      CUDA_TRY(t, launch_mixed_update(t, depth, b, k == sweeps - 1, s), "mixed update launch");
    }
  }
  // FP64 normal-equations tier for the nodes the tensor-core tier left
  // (its Gram and R live in the level's QR scratch, t->Rbuf)
  {
    ProfScope ps(K_DGRAM, s, 1, rows, 0.0);
    CUDA_TRY(t, launch_tier2_gram(t, depth, b, s), "FP64 Gram launch");
  }
  {
    ProfScope ps(K_DFACTOR, s, 1, nodes, 0.0);
    CUDA_TRY(t, launch_tier2_factor(t, depth, b, s), "FP64 factor launch");
  }
  for (int k = 0; k < sweeps; ++k) {
    {
      ProfScope ps(K_MSRESID, s, 1, rows, 0.0);
      CUDA_TRY(t, launch_tier2_sweep(t, depth, b, 0, false, s), "FP64 sweep residual launch");
    }
    {
      ProfScope ps(K_DPROJ, s, 1, rows, 0.0);
      CUDA_TRY(t, launch_tier2_sweep(t, depth, b, 1, false, s), "FP64 projection launch");
    }
    {
      ProfScope ps(K_DUPDATE, s, 1, nodes, 0.0);
      CUDA_TRY(t, launch_tier2_sweep(t, depth, b, 2, k == sweeps - 1, s), "FP64 update launch");
    }
  }
  return FMT_OK;
}

// The launches of one level step (Alg. 2 for every node of the level, then
// the octant statistics and the cumulative polynomials), all on stream s.
fmt_status fit_level_launches(fmt_tree* t, int depth, cudaStream_t s) {
  const fmt_level& L = t->lv[depth];
  const double dm = (double)L.max_m, rows = (double)L.n_points;
  if (t->P.precision == FMT_MIXED) TRY(fit_level_mixed(t, depth, s));
  {
    // Householder on [Lambda | r]: 2 m^2 flops per row (m = nmono + 1 of the row's node);
    // on the mixed path only the nodes it left to FP64 are factorised here
    // one launch per degree present in the level (launch_tile_qr)
    const int nlaunch = L.deg_mask ? __builtin_popcountll((unsigned long long)L.deg_mask) : 1;
    int mode = 0;
    if (t->piv_pending) {  // the early refits (fit_level_mixed) are done before the rest
      CUDA_TRY(t, cudaStreamWaitEvent(s, t->piv_join, 0), "early refit join");
      t->piv_pending = false;
      mode = 2;
    }
    ProfScope ps(K_TILE_QR, s, nlaunch, rows, t->P.precision == FMT_MIXED ? 0.0 : L.qr_flops);
    CUDA_TRY(t, launch_tile_qr(t, depth, t->Rbuf, s, mode), "tile QR launch");
  }
  int levels = 0;
  while ((int64_t(1) << levels) < L.max_chunks) ++levels;
  for (int tl = 0; tl < levels; ++tl) {
    // a merge of two triangles costs (2/3) m^3 flops; n_items - n_nodes merges in all
    const double pairs = tl == 0 ? (double)(L.n_items - L.n_nodes) : 0.0;
    ProfScope ps(K_COMBINE, s, 1, pairs, pairs * (2.0 / 3.0) * dm * dm * dm);
    CUDA_TRY(t, launch_combine(t, depth, tl, t->Rbuf, s), "combine launch");
  }
  {
    ProfScope ps(K_BACKSOLVE, s, 1, (double)L.n_nodes, (double)L.n_nodes * (dm - 1) * (dm - 1));
    CUDA_TRY(t, launch_backsolve(t, depth, t->Rbuf, s), "back-solve launch");
  }
  if (t->P.precision == FMT_MIXED) {
    // double-float Horner for the degrees of the tensor-core tier, FP64 above
    ProfScope ps(K_RESIDUAL, s, 2, rows, L.horner_flops);
    CUDA_TRY(t, launch_mixed_final_residual(t, depth, t->mx, s), "residual launch");
    if (t->max_degree > FMT_MIXED_MAX_DEGREE)
      CUDA_TRY(t, launch_residual(t, depth, s, FMT_MIXED_MAX_DEGREE + 1), "residual launch");
  } else {
    ProfScope ps(K_RESIDUAL, s, 1, rows, L.horner_flops);
    CUDA_TRY(t, launch_residual(t, depth, s), "residual launch");
  }
  {
    ProfScope ps(K_CHILD, s, 2, rows, 2.0 * rows);
    CUDA_TRY(t, launch_child_stats(t, depth, s), "child statistics launch");
  }
  {
    ProfScope ps(K_HCOEF, s, 1, (double)L.n_nodes, 0.0);
    CUDA_TRY(t, launch_make_cum(t, depth, s), "cumulative polynomials launch");
  }
  return FMT_OK;
}

// Graph form of a level step: the launches are captured on a private stream
// of this host thread and replayed on s.  The executable graph of each
// (device, depth) is kept per thread and updated in place when the captured
// structure matches (same kernels, same node count), else re-instantiated.
struct GraphSlots {
  cudaStream_t stream[64] = {};
  cudaGraphExec_t exec[64][FMT_MAX_DEPTH + 1] = {};
  ~GraphSlots() {
    for (int d = 0; d < 64; ++d) {
      for (int l = 0; l <= FMT_MAX_DEPTH; ++l)
        if (exec[d][l]) cudaGraphExecDestroy(exec[d][l]);
      if (stream[d]) cudaStreamDestroy(stream[d]);
    }
  }
};
thread_local GraphSlots g_graphs;

fmt_status fit_level_graph(fmt_tree* t, int depth, cudaStream_t s) {
  const int dev = t->device;
  cudaStream_t& cs = g_graphs.stream[dev];
  if (!cs) CUDA_TRY(t, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
  CUDA_TRY(t, cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed), "begin capture");
  const fmt_status st = fit_level_launches(t, depth, cs);
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(cs, &g);
  if (st != FMT_OK) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return st;
  }
  if (ce != cudaSuccess || !g) return set_err(t, FMT_ECUDA, "end capture: %s", cudaGetErrorString(ce));
  cudaGraphExec_t& ex = g_graphs.exec[dev][depth];
  bool reused = false;
  if (ex) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(ex, g, &info) == cudaSuccess) {
      reused = true;
    } else {
      cudaGetLastError();
      cudaGraphExecDestroy(ex);
      ex = nullptr;
    }
  }
  if (!ex) {
    const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
    if (ie != cudaSuccess) {
      ex = nullptr;
      cudaGraphDestroy(g);
      return set_err(t, FMT_ECUDA, "graph instantiate: %s", cudaGetErrorString(ie));
    }
  }
  cudaGraphDestroy(g);
  {
    ProfScope ps(K_GRAPH, s, 1, reused ? 1.0 : 0.0, 0.0);
    CUDA_TRY(t, cudaGraphLaunch(ex, s), "graph launch");
  }
  return FMT_OK;
}

}  // namespace

const char* check_site_name(int site) {
  static const char* const kNames[CK_SITES] = {
      "none",
      "build (k_morton, k_radix_scatter, k_gather): point index",
      "plan (k_plan_root, k_refine): node problem or rows",
      "tile QR (k_tile_qr): work item",
      "merge (k_merge, k_merge_cl, k_combine): item pair",
      "back substitution (k_backsolve): node",
      "residual (k_residual): work item",
      "child statistics (k_child_bounds, k_child_sums): rows",
      "mixed path per item (k_mbox, k_mgram, k_msresid, k_dgram, k_dproj)",
      "mixed path per node (k_mreduce, k_mfactor, k_mupdate, k_dfactor, k_dupdate)",
      "evaluation (k_evaluate): node degree",
      "cumulative polynomials (k_make_cum, k_make_hcoef): node",
      "allocation-free fit (k_fit_node_static): degree or size",
      "fmt_check_probe: index outside [0, n)"};
  return site > 0 && site < CK_SITES ? kNames[site] : "unknown site";
}

// Checked build: wait for the call's work (every stream of the tree), read
// every translation unit's check word and report the first failed site.
// While s is being captured nothing has run yet, and nothing is read.
fmt_status check_end(fmt_tree* t, cudaStream_t s) {
#ifdef FMT_CHECKED
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return FMT_OK;
  const cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return set_err(t, FMT_ECUDA, "synchronise: %s", cudaGetErrorString(e));
  // each translation unit keeps its first failed site; all of them are named
  int (*const readers[])() = {check_site_build, check_site_plan, check_site_fit, check_site_mixed};
  int sites[4], n_failed = 0;
  for (auto rd : readers) {
    const int v = rd();
    if (v < 0) return set_err(t, FMT_ECUDA, "reading a bounds-check word failed");
    if (v > 0) sites[n_failed++] = v;
  }
  if (n_failed == 1) return set_err(t, FMT_EINTERNAL, "bounds check failed: %s", check_site_name(sites[0]));
  if (n_failed > 1) {
    char buf[256];
    int o = snprintf(buf, sizeof(buf), "bounds checks failed:");
    for (int i = 0; i < n_failed && o < (int)sizeof(buf); ++i)
      o += snprintf(buf + o, sizeof(buf) - o, "%s %s", i ? ";" : "", check_site_name(sites[i]));
    return set_err(t, FMT_EINTERNAL, "%s", buf);
  }
#else
  (void)t;
  (void)s;
#endif
  return FMT_OK;
}

// error reporting for entry points defined in other translation units
fmt_status fmt_set_error(fmt_status st, const char* msg) { return set_err(nullptr, st, "%s", msg); }

extern "C" {

int32_t fmt_nmono(int32_t degree) {
  if (degree < 0) return 0;
  return (degree + 1) * (degree + 2) * (degree + 3) / 6;
}

const char* fmt_last_error(const fmt_tree* tree) { return tree ? tree->msg : g_msg; }

fmt_status oct_build(const fmt_params* params, int64_t n, const double* x, const double* y, const double* z,
                     const double* f, void* stream, fmt_tree** out) {
  if (out) *out = nullptr;
  if (params && (params->degree < 0 || params->degree > FMT_MAX_DEGREE))
    return set_err(nullptr, FMT_EINVAL, "degree %d outside [0, %d]", params->degree, FMT_MAX_DEGREE);
  if (n < 1 || n > (int64_t)0xfffffffe) return set_err(nullptr, FMT_EINVAL, "n = %lld outside [1, 2^32-2]", (long long)n);
  const int64_t offsets[2] = {0, n};
  return build_forest(params, 1, offsets, nullptr, nullptr, x, y, z, f, (cudaStream_t)stream, out);
}

fmt_status oct_build_batch(const fmt_params* params, int64_t n_problems, const int64_t* offsets,
                           const int32_t* degrees, const double* boxes, const double* x, const double* y,
                           const double* z, const double* f, void* stream, fmt_tree** out) {
  return build_forest(params, n_problems, offsets, degrees, boxes, x, y, z, f, (cudaStream_t)stream, out);
}

fmt_status fit_level(fmt_tree* t, int32_t depth, void* stream) {
  TRY(check_tree(t));
  cudaStream_t s = (cudaStream_t)stream;
  t->stream = s;
  if (t->imported) return set_err(t, FMT_EINVAL, "fit_level on an imported (evaluation-only) tree");
  if (t->done || depth != t->next_fit)
    return set_err(t, FMT_EINVAL, "fit_level(%d) out of order (expected %d)", depth, t->done ? -1 : t->next_fit);
  fmt_level& L = t->lv[depth];
  const size_t need = (size_t)L.r_total;
  if (need > t->Rbuf_cap) {
    if (t->Rbuf) tfree_one(t, t->Rbuf, s);
    t->Rbuf = nullptr;
    t->Rbuf_cap = 0;
    TRY(talloc(t, &t->Rbuf, (int64_t)need, s));
    t->Rbuf_cap = need;
  }
  if (t->P.precision == FMT_MIXED) TRY(ensure_mixed(t, depth, s));  // allocations precede any capture
  if (t->P.options & FMT_OPT_GRAPH)
    TRY(fit_level_graph(t, depth, s));
  else
    TRY(fit_level_launches(t, depth, s));
  L.fitted = true;
  t->next_fit = -1;
  t->next_refine = depth;
  return check_end(t, s);
}

fmt_status refine(fmt_tree* t, int32_t depth, int64_t* n_new_nodes, void* stream) {
  TRY(check_tree(t));
  cudaStream_t s = (cudaStream_t)stream;
  t->stream = s;
  if (!n_new_nodes) return set_err(t, FMT_EINVAL, "n_new_nodes is NULL");
  *n_new_nodes = 0;
  if (t->imported) return set_err(t, FMT_EINVAL, "refine on an imported (evaluation-only) tree");
  if (depth != t->next_refine)
    return set_err(t, FMT_EINVAL, "refine(%d) out of order (expected %d)", depth, t->next_refine);
  const fmt_level& L = t->lv[depth];
  const bool deep_ok = depth + 1 <= t->P.max_depth && depth + 1 <= FMT_MAX_DEPTH;
  if (deep_ok) {
    int64_t cap = t->n / nmin_of(t) + 1;
    if (cap > 8 * L.n_nodes) cap = 8 * L.n_nodes;
    if (cap < 1) cap = 1;
    fmt_level& N = t->lv[depth + 1];
    if (N.cap_nodes < cap) TRY(alloc_level(t, depth + 1, cap, cap + t->n / min_chunk(t) + 2, s));
  }
  {
    ProfScope ps(K_REFINE, s, 1, (double)L.n_nodes, 0.0);
    CUDA_TRY(t, launch_refine(t, depth, t->P.chunk_rows, t->chunk_floor, t->d_plan, s), "refine launch");
  }
  TRY(read_plan(t, s));
  const fmt_plan_out& pl = *t->h_plan;
  if (pl.err & FMT_ERR_TIMEOUT)
    return set_err(t, FMT_ETIMEOUT, "a tensor-core completion wait of the mixed fit timed out");
  if (pl.err) return set_err(t, FMT_EINTERNAL, "device check failed in refine (0x%llx)", (unsigned long long)pl.err);
  t->next_refine = -1;
  if (!deep_ok || pl.n_new <= 0) {
    t->done = 1;
    return check_end(t, s);
  }
  fmt_level& N = t->lv[depth + 1];
  N.n_nodes = pl.n_new;
  N.n_items = pl.n_items;
  N.max_chunks = pl.max_chunks;
  N.chunk_rows = pl.chunk_rows;
  N.n_points = pl.n_points;
  N.max_m = (int32_t)pl.max_m;
  N.deg_mask = pl.deg_mask;
  N.r_total = pl.r_total;
  N.n_hard_items = pl.n_hard_items;
  N.qr_flops = pl.qr_flops;
  N.horner_flops = pl.horner_flops;
  N.fitted = false;
  t->n_levels = depth + 2;
  t->next_fit = depth + 1;
  *n_new_nodes = pl.n_new;
  return check_end(t, s);
}

fmt_status evaluate_batch(fmt_tree* t, int64_t m, const int32_t* target_problem, const double* xq,
                          const double* yq, const double* zq, double* out, int64_t* n_outside, void* stream) {
  TRY(check_tree(t));
  cudaStream_t s = (cudaStream_t)stream;
  t->stream = s;
  if (m < 0) return set_err(t, FMT_EINVAL, "m < 0");
  if (m > 0 && (!xq || !yq || !zq || !out)) return set_err(t, FMT_EINVAL, "NULL target or output pointer");
  if (t->n_problems > 1 && m > 0 && !target_problem)
    return set_err(t, FMT_EINVAL, "a forest needs the problem of every target");
  if (!t->lv[0].fitted) return set_err(t, FMT_EINVAL, "evaluate before the roots were fitted");
  if (n_outside) *n_outside = 0;
  if (m == 0) return FMT_OK;
  if (n_outside) CUDA_TRY(t, cudaMemsetAsync(t->d_counter, 0, sizeof(unsigned long long), s), "memset");
  {
    ProfScope ps(K_EVALUATE, s, 1, (double)m, 0.0);
    CUDA_TRY(t, launch_evaluate(t, m, target_problem, xq, yq, zq, out, n_outside ? t->d_counter : nullptr, s),
             "evaluate launch");
  }
  if (n_outside) {
    unsigned long long h = 0;
    CUDA_TRY(t, cudaMemcpyAsync(&h, t->d_counter, sizeof(h), cudaMemcpyDeviceToHost, s), "copy");
    CUDA_TRY(t, cudaMemcpyAsync(t->h_err, t->d_err, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
    CUDA_TRY(t, cudaStreamSynchronize(s), "synchronise");
    if (*t->h_err & FMT_ERR_INDEX) return set_err(t, FMT_EINVAL, "target problem index out of range");
    *n_outside = (int64_t)h;
  }
  return check_end(t, s);
}

fmt_status evaluate(fmt_tree* t, int64_t m, const double* xq, const double* yq, const double* zq, double* out,
                    int64_t* n_outside, void* stream) {
  return evaluate_batch(t, m, nullptr, xq, yq, zq, out, n_outside, stream);
}

fmt_status fmt_tree_trim(fmt_tree* t, void* stream) {
  if (!t) return fmt_set_error(FMT_EINVAL, "tree is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if (t->Rbuf) tfree_one(t, t->Rbuf, s);
  t->Rbuf = nullptr;
  t->Rbuf_cap = 0;
  fmt_mixed_bufs& b = t->mx;
  void* bufs[] = {b.s, b.mstat, b.acc, b.gacc, b.dproj, b.lcoef, b.cache};
  for (void* p : bufs)
    if (p) tfree_one(t, p, s);
  b = fmt_mixed_bufs{};
  t->stream = s;
  return FMT_OK;
}

fmt_status fmt_tree_stats(fmt_tree* t, fmt_stats* o) {
  TRY(check_tree(t));
  if (!o) return set_err(t, FMT_EINVAL, "out is NULL");
  memset(o, 0, sizeof(*o));
  CUDA_TRY(t, cudaDeviceSynchronize(), "synchronise");
  o->degree = t->max_degree;
  o->nmono = t->nmono;
  o->max_depth = t->P.max_depth;
  o->n_levels = t->n_levels;
  int nf = 0;
  while (nf < t->n_levels && t->lv[nf].fitted) ++nf;
  o->n_fitted = nf;
  o->n_problems = (int32_t)t->n_problems;
  o->n_points = t->n;
  o->tau = t->tau;
  o->maxabs_f = t->maxabs;
  for (int d = 0; d < t->n_levels; ++d) {
    const fmt_level& L = t->lv[d];
    o->nodes[d] = L.n_nodes;
    o->points[d] = L.n_points;
    o->items[d] = L.n_items;
    o->chunk_rows[d] = L.chunk_rows;
    if (L.n_nodes > 0) {
      int32_t* hf = (int32_t*)malloc(sizeof(int32_t) * (size_t)L.n_nodes);
      if (!hf) return set_err(t, FMT_ENOMEM, "host allocation failed");
      cudaError_t e = cudaMemcpy(hf, L.flags, sizeof(int32_t) * (size_t)L.n_nodes, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) {
        free(hf);
        return set_err(t, FMT_ECUDA, "copy: %s", cudaGetErrorString(e));
      }
      int64_t* hc = (int64_t*)malloc(sizeof(int64_t) * (size_t)L.n_nodes);
      if (!hc) {
        free(hf);
        return set_err(t, FMT_ENOMEM, "host allocation failed");
      }
      e = cudaMemcpy(hc, L.count, sizeof(int64_t) * (size_t)L.n_nodes, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) {
        free(hf);
        free(hc);
        return set_err(t, FMT_ECUDA, "copy: %s", cudaGetErrorString(e));
      }
      for (int64_t i = 0; i < L.n_nodes; ++i) {
        o->near_tau[d] += (hf[i] & FMT_FLAG_NEAR_TAU) ? 1 : 0;
        o->rank_flagged[d] += (hf[i] & FMT_FLAG_RANK) ? 1 : 0;
        if (hf[i] & FMT_FLAG_MIXED) {
          o->mixed[d] += 1;
          o->mixed_points[d] += hc[i];
        }
      }
      free(hf);
      free(hc);
    }
  }
  return FMT_OK;
}

// bytes of the node and problem sections of an FMT2 blob
static size_t blob_node_bytes(int64_t K, int64_t nm) {
  return (size_t)K * (8 + 8 + 8 + 4 * 6 + 8 * 8 + 8 * 8 + 8 * (size_t)nm);
}
static size_t blob_problem_bytes(int64_t P) { return (size_t)P * (4 + 4 + 8 * 6 + 8 + 8); }

fmt_status fmt_tree_export(fmt_tree* t, void* host_buf, size_t* len) {
  TRY(check_tree(t));
  if (!len) return set_err(t, FMT_EINVAL, "len is NULL");
  int64_t K = 0;
  for (int d = 0; d < t->n_levels; ++d) K += t->lv[d].n_nodes;
  const int64_t nm = t->nmono, P = t->n_problems;
  const int has_pts = (t->imported || !t->x) ? 0 : 1;
  const int64_t N = has_pts ? t->n : 0;
  const size_t need =
      sizeof(fmt_export_header) + blob_node_bytes(K, nm) + blob_problem_bytes(P) + (size_t)N * (8 + 8 + 8);
  if (!host_buf) {
    *len = need;
    return FMT_OK;
  }
  if (*len < need) {
    *len = need;
    return set_err(t, FMT_EINVAL, "export buffer too small (%zu bytes needed)", need);
  }
  *len = need;
  CUDA_TRY(t, cudaDeviceSynchronize(), "synchronise");
  char* b = (char*)host_buf;
  fmt_export_header* H = (fmt_export_header*)b;
  memset(H, 0, sizeof(*H));
  H->magic = 0x32544d46u;
  H->version = 2;
  H->degree = t->max_degree;
  H->nmono = t->nmono;
  H->max_depth = t->P.max_depth;
  H->min_pts = t->P.min_pts;
  H->n_levels = t->n_levels;
  int nf = 0;
  while (nf < t->n_levels && t->lv[nf].fitted) ++nf;
  H->n_fitted = nf;
  H->has_points = has_pts;
  H->n_problems = (int32_t)P;
  H->tol_rel = t->P.tol_rel;
  H->tau = t->tau;
  H->maxabs_f = t->maxabs;
  for (int a = 0; a < 3; ++a) H->lo[a] = t->h_prob[0].lo[a];
  H->side = t->h_prob[0].side;
  H->n_points = t->n;
  H->n_nodes = K;
  for (int d = 0; d < t->n_levels; ++d) H->level_nodes[d] = t->lv[d].n_nodes;
  char* p = b + sizeof(fmt_export_header);
  uint64_t* prefix = (uint64_t*)p;
  int64_t* start = (int64_t*)(prefix + K);
  int64_t* count = start + K;
  int32_t* depth = (int32_t*)(count + K);
  int32_t* flags = depth + K;
  int32_t* deg = flags + K;
  int32_t* masks = deg + K;
  int32_t* nprob = masks + K;
  int32_t* npad = nprob + K;
  double* cE = (double*)(npad + K);
  int64_t* cn = (int64_t*)(cE + 8 * K);
  double* coef = (double*)(cn + 8 * K);
  char* pp = (char*)(coef + nm * K);
  int64_t off = 0;
  for (int d = 0; d < t->n_levels; ++d) {
    const fmt_level& L = t->lv[d];
    const size_t k = (size_t)L.n_nodes;
    if (!k) continue;
    CUDA_TRY(t, cudaMemcpy(prefix + off, L.prefix, 8 * k, cudaMemcpyDeviceToHost), "copy");
    CUDA_TRY(t, cudaMemcpy(start + off, L.start, 8 * k, cudaMemcpyDeviceToHost), "copy");
    CUDA_TRY(t, cudaMemcpy(count + off, L.count, 8 * k, cudaMemcpyDeviceToHost), "copy");
    CUDA_TRY(t, cudaMemcpy(flags + off, L.flags, 4 * k, cudaMemcpyDeviceToHost), "copy");
    CUDA_TRY(t, cudaMemcpy(deg + off, L.deg_used, 4 * k, cudaMemcpyDeviceToHost), "copy");
    CUDA_TRY(t, cudaMemcpy(masks + off, L.masks, 4 * k, cudaMemcpyDeviceToHost), "copy");
    CUDA_TRY(t, cudaMemcpy(nprob + off, L.prob, 4 * k, cudaMemcpyDeviceToHost), "copy");
    CUDA_TRY(t, cudaMemcpy(cE + 8 * off, L.child_E, 64 * k, cudaMemcpyDeviceToHost), "copy");
    CUDA_TRY(t, cudaMemcpy(cn + 8 * off, L.child_n, 64 * k, cudaMemcpyDeviceToHost), "copy");
    CUDA_TRY(t, cudaMemcpy(coef + nm * off, L.coef, 8 * nm * k, cudaMemcpyDeviceToHost), "copy");
    for (size_t i = 0; i < k; ++i) {
      depth[off + i] = d;
      npad[off + i] = 0;
    }
    if (!L.fitted) {  // nodes created by refine but not fitted yet carry no coefficients
      memset(coef + nm * off, 0, 8 * nm * k);
      memset(cE + 8 * off, 0, 64 * k);
      memset(cn + 8 * off, 0, 64 * k);
      for (size_t i = 0; i < k; ++i) deg[off + i] = -1;
    }
    off += (int64_t)k;
  }
  // problem table: degree, q_root, tau, maxabs, lo[3], side, start, count
  int32_t* pdeg = (int32_t*)pp;
  int32_t* pq = pdeg + P;
  double* ptau = (double*)(pq + P);
  double* pmax = ptau + P;
  double* plo = pmax + P;
  double* pside = plo + 3 * P;
  int64_t* pstart = (int64_t*)(pside + P);
  int64_t* pcount = pstart + P;
  for (int64_t i = 0; i < P; ++i) {
    const fmt_problem& pr = t->h_prob[i];
    pdeg[i] = pr.degree;
    pq[i] = pr.q_root;
    ptau[i] = pr.tau;
    pmax[i] = pr.maxabs;
    for (int a = 0; a < 3; ++a) plo[3 * i + a] = pr.lo[a];
    pside[i] = pr.side;
    pstart[i] = pr.start;
    pcount[i] = pr.count;
  }
  char* pts = (char*)(pcount + P);
  if (has_pts) {
    uint64_t* code = (uint64_t*)pts;
    int64_t* perm = (int64_t*)(code + N);
    double* resid = (double*)(perm + N);
    CUDA_TRY(t, cudaMemcpy(code, t->code, 8 * (size_t)N, cudaMemcpyDeviceToHost), "copy");
    uint32_t* p32 = (uint32_t*)malloc(4 * (size_t)N);
    double* rs = (double*)malloc(8 * (size_t)N);
    if (!p32 || !rs) {
      free(p32);
      free(rs);
      return set_err(t, FMT_ENOMEM, "host allocation failed");
    }
    cudaError_t e1 = cudaMemcpy(p32, t->perm, 4 * (size_t)N, cudaMemcpyDeviceToHost);
    cudaError_t e2 = cudaMemcpy(rs, t->r, 8 * (size_t)N, cudaMemcpyDeviceToHost);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
      free(p32);
      free(rs);
      return set_err(t, FMT_ECUDA, "copy failed");
    }
    for (int64_t i = 0; i < N; ++i) {
      perm[i] = p32[i];
      resid[p32[i]] = rs[i];
    }
    free(p32);
    free(rs);
  }
  return FMT_OK;
}

fmt_status fmt_tree_import(const void* host_buf, size_t len, void* stream, fmt_tree** out) {
  if (!out) return set_err(nullptr, FMT_EINVAL, "out is NULL");
  *out = nullptr;
  if (!host_buf || len < sizeof(fmt_export_header)) return set_err(nullptr, FMT_EINVAL, "blob too small");
  const fmt_export_header* H = (const fmt_export_header*)host_buf;
  if (H->magic != 0x32544d46u || H->version != 2) return set_err(nullptr, FMT_EINVAL, "not an FMT2 blob");
  if (H->degree < 0 || H->degree > FMT_MAX_DEGREE || H->nmono != fmt_nmono(H->degree) || H->n_levels < 1 ||
      H->n_levels > FMT_MAX_DEPTH + 1 || H->n_nodes < 1 || H->n_problems < 1)
    return set_err(nullptr, FMT_EINVAL, "inconsistent blob header");
  const int64_t K = H->n_nodes, nm = H->nmono, P = H->n_problems;
  // bound the counts by the bytes present before any product or sum of them,
  // so that a corrupt header cannot wrap the size check below
  const size_t body = len - sizeof(fmt_export_header);
  if ((uint64_t)K > body / blob_node_bytes(1, nm) || (uint64_t)P > body / blob_problem_bytes(1))
    return set_err(nullptr, FMT_EINVAL, "blob truncated");
  int64_t sumk = 0;
  for (int d = 0; d < H->n_levels; ++d) {
    if (H->level_nodes[d] < 1) return set_err(nullptr, FMT_EINVAL, "empty level %d in blob", d);
    if (H->level_nodes[d] > K) return set_err(nullptr, FMT_EINVAL, "level %d larger than the blob", d);
    sumk += H->level_nodes[d];
  }
  if (sumk != K) return set_err(nullptr, FMT_EINVAL, "level sizes do not add up");
  const size_t need = sizeof(fmt_export_header) + blob_node_bytes(K, nm) + blob_problem_bytes(P);
  if (len < need) return set_err(nullptr, FMT_EINVAL, "blob truncated");
  const char* p = (const char*)host_buf + sizeof(fmt_export_header);
  const uint64_t* prefix = (const uint64_t*)p;
  const int64_t* start = (const int64_t*)(prefix + K);
  const int64_t* count = start + K;
  const int32_t* depth = (const int32_t*)(count + K);
  const int32_t* flags = depth + K;
  const int32_t* deg = flags + K;
  const int32_t* masks = deg + K;
  const int32_t* nprob = masks + K;
  const int32_t* npad = nprob + K;
  const double* cE = (const double*)(npad + K);
  const int64_t* cn = (const int64_t*)(cE + 8 * K);
  const double* coef = (const double*)(cn + 8 * K);
  const char* pp = (const char*)(coef + nm * K);
  const int32_t* pdeg = (const int32_t*)pp;
  const int32_t* pq = pdeg + P;
  const double* ptau = (const double*)(pq + P);
  const double* pmax = ptau + P;
  const double* plo = pmax + P;
  const double* pside = plo + 3 * P;
  const int64_t* pstart = (const int64_t*)(pside + P);
  const int64_t* pcount = pstart + P;
  for (int64_t i = 0; i < P; ++i) {
    if (pdeg[i] < 0 || pdeg[i] > H->degree) return set_err(nullptr, FMT_EINVAL, "problem degree out of range");
    TRY(validate_box(plo[3 * i], plo[3 * i + 1], plo[3 * i + 2], pside[i]));
  }
  for (int64_t i = 0; i < K; ++i)
    if (nprob[i] < 0 || nprob[i] >= P) return set_err(nullptr, FMT_EINVAL, "node problem out of range");
  {
    int64_t o = 0;  // first node of level d
    for (int d = 0; d < H->n_levels; ++d) {
      for (int64_t i = 0; i < H->level_nodes[d]; ++i)
        if (depth[o + i] != d || (i > 0 && prefix[o + i] <= prefix[o + i - 1]))
          return set_err(nullptr, FMT_EINVAL, "blob level %d is not sorted by node key", d);
      o += H->level_nodes[d];
    }
  }
  // the blob is consistent: only now touch the device
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return set_err(nullptr, FMT_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(ce));
  TRY(device_init(dev));
  cudaStream_t s = (cudaStream_t)stream;

  fmt_tree* t = new (std::nothrow) fmt_tree();
  if (!t) return set_err(nullptr, FMT_ENOMEM, "host allocation failed");
  t->imported = true;
  t->device = dev;
  t->stream = s;
  t->P.degree = H->degree;
  t->P.max_depth = H->max_depth;
  t->P.min_pts = H->min_pts;
  t->P.precision = FMT_FP64;
  t->P.tol_rel = H->tol_rel;
  for (int a = 0; a < 3; ++a) t->P.lo[a] = H->lo[a];
  t->P.side = H->side;
  t->nmono = (int32_t)nm;
  t->max_degree = H->degree;
  t->n = H->n_points;
  t->n_problems = P;
  t->tau = H->tau;
  t->maxabs = H->maxabs_f;
  t->h_prob = (fmt_problem*)calloc((size_t)P, sizeof(fmt_problem));
  if (!t->h_prob) {
    destroy(t);
    return set_err(nullptr, FMT_ENOMEM, "host allocation failed");
  }
  for (int64_t i = 0; i < P; ++i) {
    fmt_problem& pr = t->h_prob[i];
    pr.degree = pdeg[i];
    pr.q_root = pq[i];
    pr.tau = ptau[i];
    pr.maxabs = pmax[i];
    for (int a = 0; a < 3; ++a) pr.lo[a] = plo[3 * i + a];
    pr.side = pside[i];
    pr.S = 2097152.0 / pr.side;
    pr.inv_side = 1.0 / pr.side;
    for (int a = 0; a < 3; ++a) pr.hi[a] = pr.lo[a] + pr.side;
    pr.start = pstart[i];
    pr.count = pcount[i];
  }
  fmt_status st = FMT_OK;
  if ((st = talloc(t, &t->d_err, 1, s)) || (st = talloc(t, &t->d_counter, 1, s)) ||
      (st = talloc(t, &t->d_plan, 1, s)) || (st = talloc(t, &t->d_prob, P, s))) {
    destroy(t);
    return st;
  }
  if (cudaMallocHost((void**)&t->h_err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    destroy(t);
    return set_err(nullptr, FMT_ENOMEM, "pinned host allocation failed");
  }
  cudaError_t e0 = cudaMemcpyAsync(t->d_prob, t->h_prob, sizeof(fmt_problem) * (size_t)P, cudaMemcpyHostToDevice, s);
  if (e0 == cudaSuccess) e0 = cudaMemsetAsync(t->d_err, 0, sizeof(int), s);
  if (e0 != cudaSuccess) {
    destroy(t);
    return set_err(nullptr, FMT_ECUDA, "import upload: %s", cudaGetErrorString(e0));
  }
  int64_t off = 0;
  for (int d = 0; d < H->n_levels; ++d) {
    const int64_t k = H->level_nodes[d];
    if ((st = alloc_level(t, d, k, 1, s))) {
      destroy(t);
      return st;
    }
    fmt_level& L = t->lv[d];
    L.n_nodes = k;
    L.fitted = true;
    cudaError_t e = cudaSuccess;
    if ((e = cudaMemcpyAsync(L.prefix, prefix + off, 8 * k, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(L.prob, nprob + off, 4 * k, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(L.start, start + off, 8 * k, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(L.count, count + off, 8 * k, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(L.flags, flags + off, 4 * k, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(L.deg_used, deg + off, 4 * k, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(L.masks, masks + off, 4 * k, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(L.child_E, cE + 8 * off, 64 * k, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(L.child_n, cn + 8 * off, 64 * k, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(L.coef, coef + nm * off, 8 * nm * k, cudaMemcpyHostToDevice, s)) != cudaSuccess) {
      destroy(t);
      return set_err(nullptr, FMT_ECUDA, "import upload: %s", cudaGetErrorString(e));
    }
    {
      ProfScope ps(K_HCOEF, s, 2, (double)k, 0.0);
      e = launch_make_hcoef(t, d, s);
      if (e == cudaSuccess) e = launch_make_cum(t, d, s);
    }
    if (e != cudaSuccess) {
      destroy(t);
      return set_err(nullptr, FMT_ECUDA, "import upload: %s", cudaGetErrorString(e));
    }
    off += k;
  }
  t->n_levels = H->n_levels;
  t->done = 1;
  t->next_fit = -1;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    destroy(t);
    return set_err(nullptr, FMT_ECUDA, "synchronise: %s", cudaGetErrorString(e));
  }
  if (check_end(t, s) != FMT_OK) {
    set_err(nullptr, FMT_EINTERNAL, "%s", t->msg);
    destroy(t);
    return FMT_EINTERNAL;
  }
  *out = t;
  return FMT_OK;
}

void fmt_tree_free(fmt_tree* t) { destroy(t); }

fmt_status fmt_profile_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(g_pmu);
  if (on) {
    for (int64_t i = 0; i < g_nrecs; ++i) {
      cudaEventDestroy(g_recs[i].a);
      cudaEventDestroy(g_recs[i].b);
    }
    g_nrecs = 0;
    for (int k = 0; k < FMT_PROFILE_CLASSES; ++k) {
      g_launch[k] = 0;
      g_units[k] = 0.0;
      g_flops[k] = 0.0;
    }
  }
  g_prof_on = on != 0;
  return FMT_OK;
}

fmt_status fmt_profile_read(fmt_profile* out) {
  if (!out) return set_err(nullptr, FMT_EINVAL, "out is NULL");
  memset(out, 0, sizeof(*out));
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return set_err(nullptr, FMT_ECUDA, "synchronise: %s", cudaGetErrorString(e));
  std::lock_guard<std::mutex> lk(g_pmu);
  for (int k = 0; k < FMT_PROFILE_CLASSES; ++k) {
    out->launches[k] = g_launch[k];
    out->units[k] = g_units[k];
    out->flops[k] = g_flops[k];
  }
  for (int64_t i = 0; i < g_nrecs; ++i) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, g_recs[i].a, g_recs[i].b) == cudaSuccess) out->ms[g_recs[i].k] += ms;
    else cudaGetLastError();
  }
  return FMT_OK;
}

fmt_status fmt_probe_dfma(int64_t iters, double* dfma_per_s, void* stream) {
  if (!dfma_per_s || iters < 1) return set_err(nullptr, FMT_EINVAL, "bad probe arguments");
  *dfma_per_s = 0.0;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = (nsm > 0 ? nsm : 152) * 4;  // 32 warps per SM
  double* buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * (size_t)blocks * 256) != cudaSuccess) {
    cudaGetLastError();
    return set_err(nullptr, FMT_ENOMEM, "probe buffer allocation failed");
  }
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaError_t e = launch_probe_dfma(iters / 8 + 1, blocks, buf, s);  // warm-up
  float best = 0.0f;
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
    cudaEventRecord(a, s);
    e = launch_probe_dfma(iters, blocks, buf, s);
    cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess && (best == 0.0f || ms < best)) best = ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(buf);
  if (e != cudaSuccess) return set_err(nullptr, FMT_ECUDA, "probe: %s", cudaGetErrorString(e));
  *dfma_per_s = 8.0 * (double)iters * blocks * 256.0 / (best * 1e-3);
  return FMT_OK;
}

const char* fmt_profile_class_name(int32_t k) { return (k >= 0 && k < K_NCLASS) ? kClassNames[k] : nullptr; }

}  // extern "C"

extern "C" fmt_status fmt_debug_fail_alloc(int64_t k) {
  if (k < 0) return set_err(nullptr, FMT_EINVAL, "fmt_debug_fail_alloc: k < 0");
  g_fail_alloc.store(k);
  return FMT_OK;
}

extern "C" fmt_status fmt_wait_probe(int64_t limit_ns, void* stream) {
  if (limit_ns < 1000 || limit_ns > 10000000000ll)
    return set_err(nullptr, FMT_EINVAL, "fmt_wait_probe: limit_ns outside [1e3, 1e10]");
  cudaStream_t s = (cudaStream_t)stream;
  int* d_err = nullptr;
  int h_err = 0;
  cudaError_t e = cudaMalloc(&d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = launch_wait_probe((unsigned long long)limit_ns, d_err, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (d_err) cudaFree(d_err);
  if (e != cudaSuccess) return set_err(nullptr, FMT_ECUDA, "fmt_wait_probe: %s", cudaGetErrorString(e));
  if (h_err & FMT_ERR_TIMEOUT)
    return set_err(nullptr, FMT_ETIMEOUT, "bounded mbarrier wait ran out after %lld ns", (long long)limit_ns);
  return FMT_OK;
}

extern "C" int32_t fmt_checked_build(void) {
#ifdef FMT_CHECKED
  return 1;
#else
  return 0;
#endif
}

extern "C" fmt_status fmt_check_probe(int32_t i, int32_t n, void* stream) {
  if (i < 0 || i >= 64 || n < 0 || n > 32)
    return set_err(nullptr, FMT_EINVAL, "fmt_check_probe: i outside [0, 64) or n outside [0, 32]");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_check_probe(i, n, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_err(nullptr, FMT_ECUDA, "fmt_check_probe: %s", cudaGetErrorString(e));
  return check_end(nullptr, s);
}

extern "C" fmt_status fmt_debug_item_rows(fmt_tree* t, int32_t depth, int64_t item, int64_t start, int64_t end,
                                          void* stream) {
  TRY(check_tree(t));
  cudaStream_t s = (cudaStream_t)stream;
  if (t->imported || t->done || depth != t->next_fit)
    return set_err(t, FMT_EINVAL, "fmt_debug_item_rows: depth %d is not the planned level awaiting its fit", depth);
  const fmt_level& L = t->lv[depth];
  if (item < 0 || item >= L.n_items) return set_err(t, FMT_EINVAL, "fmt_debug_item_rows: item out of range");
  if (start < 0 || start > end || end > t->n)
    return set_err(t, FMT_EINVAL, "fmt_debug_item_rows: rows outside [0, n]");
  const int64_t v[2] = {start, end};
  cudaError_t e = cudaMemcpyAsync(L.item_start + item, &v[0], sizeof(int64_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(L.item_end + item, &v[1], sizeof(int64_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // v lives on this stack
  if (e != cudaSuccess) return set_err(t, FMT_ECUDA, "fmt_debug_item_rows: %s", cudaGetErrorString(e));
  return FMT_OK;
}
