// fmt_serve.cu -- a serving engine over the four calls of the method:
// fit+evaluate requests of very different sizes are queued, admitted against
// a device-memory budget and run by worker slots (one host thread and one
// CUDA stream each).  A slot that frees up forms its next batch from the
// queue -- the oldest request and every queued request with the same batch
// key, while the batch's point cap and the budget allow -- and runs it as one
// forest (oct_build_batch, fit_level/refine per level, evaluate_batch), so
// requests that arrive while other batches are on the GPU join the next
// batch, and batches of different slots overlap on the device (continuous
// batching).  The paper has no serving counterpart; every numerical step is
// the library's own.

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

struct Req {
  fmt_request r;
  int64_t ticket = 0;
  double est = 0.0;  // admission estimate, bytes
  fmt_request_result res{};
  bool done = false;
};

// Requests of one batch must agree on the parameters the forest shares.
bool same_key(const fmt_params& a, const fmt_params& b) {
  return a.precision == b.precision && a.max_depth == b.max_depth && a.min_pts == b.min_pts &&
         a.tol_rel == b.tol_rel && a.sweeps == b.sweeps && a.chunk_rows == b.chunk_rows;
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

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) cap = bytes;
    return e;
  }
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

}  // namespace

struct fmt_server {
  int device = 0;
  double budget = 0.0, admitted = 0.0;
  int64_t max_batch_points = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Req>> queue;
  std::unordered_map<int64_t, std::shared_ptr<Req>> tickets;
  int64_t next_ticket = 1, next_batch = 1;
  bool stop = false;
  std::vector<std::thread> slots;

  void run_slot();
  fmt_status run_batch(std::vector<std::shared_ptr<Req>>& batch, cudaStream_t s, DevBuf* bufs, int64_t batch_id);
};

void fmt_server::run_slot() {
  cudaSetDevice(device);
  cudaStream_t s = nullptr;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  DevBuf bufs[3];  // points (x,y,z,f), targets (xq,yq,zq), results + target problem ids
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
              if (same_key(q.r.params, head->r.params) && admitted + q.est <= budget &&
                  (first || pts + q.r.n <= max_batch_points)) {
                admitted += q.est;
                pts += q.r.n;
                batch.push_back(*it);
                it = queue.erase(it);
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
    const fmt_status st = run_batch(batch, s, bufs, bid);
    const double t1 = now_s();
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
        admitted -= q->est;
      }
    }
    cv_done.notify_all();
    cv_work.notify_all();
  }
  cudaStreamDestroy(s);
}

fmt_status fmt_server::run_batch(std::vector<std::shared_ptr<Req>>& batch, cudaStream_t s, DevBuf* bufs,
                                 int64_t batch_id) {
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
  if (bufs[0].ensure(sizeof(double) * 4 * (size_t)N) != cudaSuccess ||
      bufs[1].ensure(sizeof(double) * 3 * (size_t)(M > 0 ? M : 1)) != cudaSuccess ||
      bufs[2].ensure((sizeof(double) + sizeof(int32_t)) * (size_t)(M > 0 ? M : 1)) != cudaSuccess) {
    cudaGetLastError();
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
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (tree) fmt_tree_free(tree);
  if (st == FMT_OK && e != cudaSuccess) {
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
  delete sv;
  return FMT_OK;
}

}  // extern "C"
