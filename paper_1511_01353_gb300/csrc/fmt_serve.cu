// fmt_serve.cu -- a serving engine over the four calls of the method:
// fit+evaluate requests of very different sizes are queued, admitted against
// a device-memory budget and run by worker slots (one host thread and one
// CUDA stream each).  A slot that frees up forms its next batch from the
// queue -- the oldest request and every queued request with the same batch
// key (shared parameters and size class), while the batch's point cap and
// the budget allow -- and runs it as one forest (oct_build_batch,
// fit_level/refine per level, evaluate_batch), so requests that arrive while
// other batches are on the GPU join the next batch, and batches of different
// slots overlap on the device (continuous batching).  A request may keep its
// tree resident on the device; evaluate-only requests then run against it
// until it is released, and its memory stays counted against the budget.
// The paper has no serving counterpart; every numerical step is the
// library's own.

#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string.h>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "fmt_internal.cuh"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// A forest kept on the device after its batch because some of its requests
// asked to keep their trees (its fit scratch freed by fmt_tree_trim):
// evaluate-only requests run against it until the last of those requests is
// released.  `held` (the resident estimate of its requests) stays counted
// against the budget until then.
struct Resident {
  fmt_tree* tree = nullptr;
  int refs = 0;      // kept requests not yet released, plus evaluations in flight
  double held = 0.0;
  std::mutex eval_mu;  // one evaluation at a time on a tree
};
struct Handle {
  std::shared_ptr<Resident> res;
  int32_t problem = 0;
};

struct Req {
  int kind = 0;  // 0: fit (+ evaluate); 1: evaluate on a resident tree
  fmt_request r;
  int64_t ticket = 0;
  double est = 0.0;  // admission estimate, bytes
  fmt_request_result res{};
  bool done = false;
  Handle h;  // kind 1: the tree and problem
};

// Requests of one batch must agree on the parameters the forest shares and
// on their size class (decade of the point count), so that a batch of small
// requests is not held back by a large one that runs much longer.
int size_class(int64_t n) {
  int c = 0;
  while (n >= 10) {
    n /= 10;
    ++c;
  }
  return c;
}
bool same_key(const Req& a, const Req& b) {
  const fmt_params &pa = a.r.params, &pb = b.r.params;
  return a.kind == 0 && b.kind == 0 && pa.precision == pb.precision && pa.max_depth == pb.max_depth &&
         pa.min_pts == pb.min_pts && pa.tol_rel == pb.tol_rel && pa.sweeps == pb.sweeps &&
         pa.chunk_rows == pb.chunk_rows && size_class(a.r.n) == size_class(b.r.n);
}

// Device bytes a request may need while it runs: inputs, sorted copies,
// keys and sort scratch, per-level node tables, the QR or Gram scratch of a
// level (bounded per point by the chunk planner's rows >= 4m per item), and
// its targets.
// A work item holds at least nmono rows, so the m x m QR triangle costs at
// most 8 m bytes per point and the mixed path's Gram accumulator (about
// 2 m x 128 doubles per item) at most about 9 m.
double estimate_bytes(const fmt_request& r) {
  const double m = (double)fmt_nmono(r.params.degree) + 1.0;
  const double per_point = 240.0 + 8.0 * m + (r.params.precision == FMT_MIXED ? 9.0 * m : 0.0);
  return (double)r.n * per_point + (double)r.m * 48.0 + 32.0 * 1024 * 1024;
}
double estimate_eval_bytes(int64_t m) { return (double)m * 48.0 + 1024.0 * 1024; }
// A resident forest after fmt_tree_trim: sorted points, codes and
// permutation (44 B per point) and per-level node tables with their
// coefficients (bounded by about 40 B per point and level over 8 levels).
double estimate_resident_bytes(const fmt_request& r) { return (double)r.n * 400.0 + 8.0 * 1024 * 1024; }

// Staging buffers of one batch, stream-ordered pool allocations on the
// slot's stream, returned to the pool when the batch ends (nothing outside
// the admitted estimates stays allocated).
struct DevBuf {
  void* p = nullptr;
  cudaError_t alloc(size_t bytes, cudaStream_t s) { return cudaMallocAsync(&p, bytes, s); }
  void release(cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
  }
};

__global__ void k_fill_i32(int32_t* a, int64_t n, int32_t v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = v;
}

}  // namespace

struct fmt_server {
  int device = 0;
  double budget = 0.0, admitted = 0.0, peak_admitted = 0.0;
  int64_t max_batch_points = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Req>> queue;
  std::unordered_map<int64_t, std::shared_ptr<Req>> tickets;
  std::unordered_map<int64_t, Handle> residents;
  int64_t next_ticket = 1, next_batch = 1, next_resident = 1;
  bool stop = false;
  std::vector<std::thread> slots;

  void run_slot();
  fmt_status run_batch(std::vector<std::shared_ptr<Req>>& batch, cudaStream_t s, int64_t batch_id);
  fmt_status run_eval(Req& q, cudaStream_t s);
  void admit(double bytes) {  // with mu held
    admitted += bytes;
    if (admitted > peak_admitted) peak_admitted = admitted;
  }
  // Drops one reference; the caller frees the returned tree (outside mu) if
  // it was the last.  With mu held.
  fmt_tree* unref(Resident& r) {
    if (--r.refs > 0) return nullptr;
    admitted -= r.held;
    fmt_tree* t = r.tree;
    r.tree = nullptr;
    return t;
  }
};

void fmt_server::run_slot() {
  cudaSetDevice(device);
  cudaStream_t s = nullptr;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  for (;;) {
    std::vector<std::shared_ptr<Req>> batch;
    int64_t bid = 0;
    {
      std::unique_lock<std::mutex> lk(mu);
      for (;;) {
        if (stop && queue.empty()) break;
        if (!queue.empty()) {
          // the oldest request opens the batch; compatible requests behind it join while they fit
          std::shared_ptr<Req> head = queue.front();
          if (head->est > budget) {  // can never be admitted
            queue.pop_front();
            head->res.status = FMT_ENOMEM;
            head->res.t_start = head->res.t_done = now_s();
            head->done = true;
            cv_done.notify_all();
            continue;
          }
          if (admitted + head->est <= budget) {
            int64_t pts = 0;
            for (auto it = queue.begin(); it != queue.end();) {
              Req& q = **it;
              const bool first = batch.empty();
              if ((first || same_key(q, *head)) && admitted + q.est <= budget &&
                  (first || pts + q.r.n <= max_batch_points)) {
                admit(q.est);
                pts += q.r.n;
                batch.push_back(*it);
                it = queue.erase(it);
                if (q.kind == 1) break;  // an evaluation runs alone
              } else {
                ++it;
              }
            }
            bid = next_batch++;
            break;
          }
        }
        cv_work.wait(lk);
      }
    }
    if (batch.empty()) break;  // stopping
    const double t0 = now_s();
    for (auto& q : batch) q->res.t_start = t0;
    const fmt_status st = batch[0]->kind == 1 ? run_eval(*batch[0], s) : run_batch(batch, s, bid);
    const double t1 = now_s();
    fmt_tree* to_free = nullptr;
    {
      std::lock_guard<std::mutex> lk(mu);
      int64_t pts = 0;
      for (auto& q : batch) pts += q->r.n;
      for (auto& q : batch) {
        q->res.status = st;
        q->res.t_done = t1;
        q->res.batch_id = bid;
        q->res.batch_requests = (int32_t)batch.size();
        q->res.batch_points = pts;
        q->done = true;
        admitted -= q->est;  // a kept forest is held by its resident estimate instead
      }
      if (batch[0]->kind == 1) to_free = unref(*batch[0]->h.res);
    }
    if (to_free) fmt_tree_free(to_free);
    cv_done.notify_all();
    cv_work.notify_all();
  }
  cudaStreamDestroy(s);
}

fmt_status fmt_server::run_batch(std::vector<std::shared_ptr<Req>>& batch, cudaStream_t s, int64_t batch_id) {
  (void)batch_id;
  const int64_t P = (int64_t)batch.size();
  std::vector<int64_t> offsets(P + 1, 0), toff(P + 1, 0);
  std::vector<int32_t> degrees(P);
  std::vector<double> boxes(4 * P);
  for (int64_t i = 0; i < P; ++i) {
    const fmt_request& r = batch[i]->r;
    offsets[i + 1] = offsets[i] + r.n;
    toff[i + 1] = toff[i] + r.m;
    degrees[i] = r.params.degree;
    boxes[4 * i + 0] = r.params.lo[0];
    boxes[4 * i + 1] = r.params.lo[1];
    boxes[4 * i + 2] = r.params.lo[2];
    boxes[4 * i + 3] = r.params.side;
  }
  const int64_t N = offsets[P], M = toff[P];
  DevBuf bufs[3];  // points (x,y,z,f), targets (xq,yq,zq), results + target problem ids
  auto release = [&] {
    for (auto& b : bufs) b.release(s);
  };
  if (bufs[0].alloc(sizeof(double) * 4 * (size_t)N, s) != cudaSuccess ||
      bufs[1].alloc(sizeof(double) * 3 * (size_t)(M > 0 ? M : 1), s) != cudaSuccess ||
      bufs[2].alloc((sizeof(double) + sizeof(int32_t)) * (size_t)(M > 0 ? M : 1), s) != cudaSuccess) {
    cudaGetLastError();
    release();
    return FMT_ENOMEM;
  }
  double* dx = (double*)bufs[0].p;
  double *dy = dx + N, *dz = dy + N, *df = dz + N;
  double* dxq = (double*)bufs[1].p;
  double *dyq = dxq + M, *dzq = dyq + M;
  double* dout = (double*)bufs[2].p;
  int32_t* dtp = (int32_t*)(dout + (M > 0 ? M : 1));
  std::vector<int32_t> tp((size_t)M);
  for (int64_t i = 0; i < P; ++i)
    for (int64_t k = toff[i]; k < toff[i + 1]; ++k) tp[(size_t)k] = (int32_t)i;
  cudaError_t e = cudaSuccess;
  for (int64_t i = 0; i < P && e == cudaSuccess; ++i) {
    const fmt_request& r = batch[i]->r;
    const size_t nb = sizeof(double) * (size_t)r.n, mb = sizeof(double) * (size_t)r.m;
    const int64_t o = offsets[i], to = toff[i];
    if ((e = cudaMemcpyAsync(dx + o, r.x, nb, cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(dy + o, r.y, nb, cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(dz + o, r.z, nb, cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(df + o, r.f, nb, cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
    if (r.m > 0) {
      if ((e = cudaMemcpyAsync(dxq + to, r.xq, mb, cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
      if ((e = cudaMemcpyAsync(dyq + to, r.yq, mb, cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
      if ((e = cudaMemcpyAsync(dzq + to, r.zq, mb, cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
    }
  }
  if (e == cudaSuccess && M > 0)
    e = cudaMemcpyAsync(dtp, tp.data(), sizeof(int32_t) * (size_t)M, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaStreamSynchronize(s);
    release();
    return FMT_ECUDA;
  }
  fmt_params prm = batch[0]->r.params;
  fmt_tree* tree = nullptr;
  fmt_status st = oct_build_batch(&prm, P, offsets.data(), degrees.data(), boxes.data(), dx, dy, dz, df, s, &tree);
  for (int d = 0; st == FMT_OK; ++d) {
    if ((st = fit_level(tree, d, s)) != FMT_OK) break;
    int64_t nn = 0;
    if ((st = refine(tree, d, &nn, s)) != FMT_OK || nn == 0) break;
  }
  if (st == FMT_OK && M > 0) st = evaluate_batch(tree, M, dtp, dxq, dyq, dzq, dout, nullptr, s);
  if (st == FMT_OK && M > 0) {
    for (int64_t i = 0; i < P && e == cudaSuccess; ++i) {
      const fmt_request& r = batch[i]->r;
      if (r.m > 0)
        e = cudaMemcpyAsync(r.out, dout + toff[i], sizeof(double) * (size_t)r.m, cudaMemcpyDeviceToHost, s);
    }
  }
  release();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (st == FMT_OK && e != cudaSuccess) {
    cudaGetLastError();
    st = FMT_ECUDA;
  }
  // keep the forest on the device if any request asked for it
  int kept = 0;
  for (auto& q : batch) kept += q->r.keep ? 1 : 0;
  if (st == FMT_OK && kept > 0 && tree && fmt_tree_trim(tree, s) == FMT_OK) {
    auto res = std::make_shared<Resident>();
    res->tree = tree;
    res->refs = kept;
    double held = 0.0;
    for (auto& q : batch) held += estimate_resident_bytes(q->r);
    res->held = held;
    std::lock_guard<std::mutex> lk(mu);
    admit(held);  // the batch's fit estimates are returned when it completes
    for (int64_t i = 0; i < P; ++i) {
      if (!batch[i]->r.keep) continue;
      const int64_t id = next_resident++;
      residents[id] = Handle{res, (int32_t)i};
      batch[i]->res.resident_id = id;
      batch[i]->res.problem = (int32_t)i;
    }
    return st;
  }
  if (tree) fmt_tree_free(tree);
  return st;
}

// An evaluate-only request: the targets of one problem of a resident forest.
fmt_status fmt_server::run_eval(Req& q, cudaStream_t s) {
  Resident& R = *q.h.res;
  std::lock_guard<std::mutex> lk(R.eval_mu);
  const int64_t M = q.r.m;
  if (M == 0) return FMT_OK;
  DevBuf b;
  if (b.alloc((3 * sizeof(double) + sizeof(double) + sizeof(int32_t)) * (size_t)M, s) != cudaSuccess) {
    cudaGetLastError();
    return FMT_ENOMEM;
  }
  double* dxq = (double*)b.p;
  double *dyq = dxq + M, *dzq = dyq + M, *dout = dzq + M;
  int32_t* dtp = (int32_t*)(dout + M);
  const size_t mb = sizeof(double) * (size_t)M;
  cudaError_t e = cudaMemcpyAsync(dxq, q.r.xq, mb, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dyq, q.r.yq, mb, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dzq, q.r.zq, mb, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    k_fill_i32<<<(unsigned)((M + 255) / 256 < 1024 ? (M + 255) / 256 : 1024), 256, 0, s>>>(dtp, M, q.h.problem);
    e = cudaGetLastError();
  }
  fmt_status st = e == cudaSuccess ? evaluate_batch(R.tree, M, dtp, dxq, dyq, dzq, dout, nullptr, s) : FMT_ECUDA;
  if (st == FMT_OK) e = cudaMemcpyAsync(q.r.out, dout, mb, cudaMemcpyDeviceToHost, s);
  b.release(s);
  const cudaError_t e2 = cudaStreamSynchronize(s);
  if (st == FMT_OK && (e != cudaSuccess || e2 != cudaSuccess)) {
    cudaGetLastError();
    st = FMT_ECUDA;
  }
  return st;
}

extern "C" {

double fmt_server_clock(void) { return now_s(); }

fmt_status fmt_server_create(int32_t slots, double budget_bytes, int64_t max_batch_points, fmt_server** out) {
  if (!out) return fmt_set_error(FMT_EINVAL, "out is NULL");
  *out = nullptr;
  if (slots < 1 || slots > 64 || !(budget_bytes > 0.0) || max_batch_points < 1)
    return fmt_set_error(FMT_EINVAL, "server: slots in 1..64, budget_bytes > 0, max_batch_points >= 1");
  fmt_server* sv = new (std::nothrow) fmt_server();
  if (!sv) return fmt_set_error(FMT_ENOMEM, "host allocation failed");
  cudaGetDevice(&sv->device);
  sv->budget = budget_bytes;
  sv->max_batch_points = max_batch_points;
  for (int i = 0; i < slots; ++i) sv->slots.emplace_back([sv] { sv->run_slot(); });
  *out = sv;
  return FMT_OK;
}

fmt_status fmt_server_submit(fmt_server* sv, const fmt_request* r, int64_t* ticket) {
  if (!sv || !r || !ticket) return fmt_set_error(FMT_EINVAL, "server, request and ticket must not be NULL");
  const fmt_params& p = r->params;
  if (r->n < 1 || !r->x || !r->y || !r->z || !r->f || r->m < 0 || (r->m > 0 && (!r->xq || !r->yq || !r->zq || !r->out)))
    return fmt_set_error(FMT_EINVAL, "request: n >= 1 and host arrays for the points (and the m targets)");
  if (p.degree < 0 || p.degree > FMT_MAX_DEGREE || !(p.side > 0.0))
    return fmt_set_error(FMT_EINVAL, "request: degree in 0..14 and side > 0");
  if (r->keep != 0 && r->keep != 1) return fmt_set_error(FMT_EINVAL, "request: keep is 0 or 1");
  auto q = std::make_shared<Req>();
  q->r = *r;
  q->est = estimate_bytes(*r);
  q->res.t_submit = now_s();
  q->res.status = FMT_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) return fmt_set_error(FMT_EINVAL, "server is shutting down");
    q->ticket = sv->next_ticket++;
    sv->tickets[q->ticket] = q;
    sv->queue.push_back(q);
    *ticket = q->ticket;
  }
  sv->cv_work.notify_one();
  return FMT_OK;
}

fmt_status fmt_server_submit_eval(fmt_server* sv, int64_t resident_id, int64_t m, const double* xq, const double* yq,
                                  const double* zq, double* out, int64_t* ticket) {
  if (!sv || !ticket) return fmt_set_error(FMT_EINVAL, "server and ticket must not be NULL");
  if (m < 0 || (m > 0 && (!xq || !yq || !zq || !out)))
    return fmt_set_error(FMT_EINVAL, "evaluation request: m >= 0 and host arrays for the m targets");
  auto q = std::make_shared<Req>();
  q->kind = 1;
  q->r = fmt_request{};
  q->r.m = m;
  q->r.xq = xq;
  q->r.yq = yq;
  q->r.zq = zq;
  q->r.out = out;
  q->est = estimate_eval_bytes(m);
  q->res.t_submit = now_s();
  q->res.status = FMT_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) return fmt_set_error(FMT_EINVAL, "server is shutting down");
    auto it = sv->residents.find(resident_id);
    if (it == sv->residents.end()) return fmt_set_error(FMT_EINVAL, "unknown or released resident tree");
    q->h = it->second;
    q->h.res->refs += 1;  // the tree stays while the evaluation is queued or running
    q->res.resident_id = resident_id;
    q->res.problem = q->h.problem;
    q->ticket = sv->next_ticket++;
    sv->tickets[q->ticket] = q;
    sv->queue.push_back(q);
    *ticket = q->ticket;
  }
  sv->cv_work.notify_one();
  return FMT_OK;
}

fmt_status fmt_server_release(fmt_server* sv, int64_t resident_id) {
  if (!sv) return fmt_set_error(FMT_EINVAL, "server is NULL");
  fmt_tree* to_free = nullptr;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->residents.find(resident_id);
    if (it == sv->residents.end()) return fmt_set_error(FMT_EINVAL, "unknown or released resident tree");
    std::shared_ptr<Resident> res = it->second.res;
    sv->residents.erase(it);
    to_free = sv->unref(*res);
  }
  if (to_free) fmt_tree_free(to_free);
  sv->cv_work.notify_all();
  return FMT_OK;
}

fmt_status fmt_server_memory(fmt_server* sv, double* admitted, double* peak_admitted, int64_t* resident_trees) {
  if (!sv) return fmt_set_error(FMT_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(sv->mu);
  if (admitted) *admitted = sv->admitted;
  if (peak_admitted) *peak_admitted = sv->peak_admitted;
  if (resident_trees) *resident_trees = (int64_t)sv->residents.size();
  return FMT_OK;
}

fmt_status fmt_server_wait(fmt_server* sv, int64_t ticket, double timeout_s, fmt_request_result* res) {
  if (!sv || !res) return fmt_set_error(FMT_EINVAL, "server and result must not be NULL");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->tickets.find(ticket);
  if (it == sv->tickets.end()) return fmt_set_error(FMT_EINVAL, "unknown ticket");
  std::shared_ptr<Req> q = it->second;
  const auto pred = [&] { return q->done; };
  if (timeout_s < 0.0) {
    sv->cv_done.wait(lk, pred);
  } else if (!sv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) {
    return fmt_set_error(FMT_ETIMEOUT, "request not done within the timeout");
  }
  *res = q->res;
  sv->tickets.erase(ticket);
  return FMT_OK;
}

fmt_status fmt_server_destroy(fmt_server* sv) {
  if (!sv) return fmt_set_error(FMT_EINVAL, "server is NULL");
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  for (auto& t : sv->slots) t.join();
  // trees still resident go with the server
  std::vector<fmt_tree*> trees;
  for (auto& kv : sv->residents)
    if (kv.second.res->tree) {
      trees.push_back(kv.second.res->tree);
      kv.second.res->tree = nullptr;
    }
  for (fmt_tree* t : trees) fmt_tree_free(t);
  delete sv;
  return FMT_OK;
}

}  // extern "C"
