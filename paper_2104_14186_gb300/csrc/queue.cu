// Request queue with HBM-budget admission and continuous batching, and the batched
// solver built on it.  Not part of the paper's method: a serving layer around
// qdwhp_eig / qdwhp_svd.
//
// A queue owns `max_slots` worker threads, each with its own CUDA stream, and one
// device allocation of `hbm_budget_bytes` that it sub-allocates (first fit) as
// workspaces.  A submitted request records an event on the caller's stream (its input
// is ready when that event completes) and joins a FIFO.  A free worker takes the
// oldest pending request whose workspace fits in the free part of the pool, so
// requests that arrive while others run start as soon as a slot and memory free up;
// their kernels overlap on the device through the workers' streams.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <algorithm>

#include "internal.h"

struct qdwhp_queue;

namespace qdwhp {

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, cap); offsets are 256-byte aligned.
class Pool {
 public:
  explicit Pool(size_t cap) { free_[0] = cap; }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) & ~size_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_[*off] = bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off) {
    auto u = used_.find(off);
    if (u == used_.end()) return;
    size_t start = off, len = u->second;
    used_.erase(u);
    auto next = free_.lower_bound(start);
    if (next != free_.end() && next->first == start + len) {
      len += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == start) {
        start = prev->first;
        len += prev->second;
        free_.erase(prev);
      }
    }
    free_[start] = len;
  }

 private:
  std::map<size_t, size_t> free_, used_;
};

struct Request {
  uint64_t id = 0;
  bool svd = false;
  const double* A = nullptr;
  int64_t m = 0, n = 0, lda = 0, k = 0;
  qdwhp_opts opts;
  double *vals = nullptr, *U = nullptr, *V = nullptr;
  int64_t ldu = 0, ldv = 0;
  size_t ws_bytes = 0;
  cudaEvent_t ready = nullptr;
  qdwhp_status status = QDWHP_PENDING;
  qdwhp_info info;
  double t_submit = 0, t_start = 0, t_done = 0;
  bool done = false;
};

}  // namespace

}  // namespace qdwhp

struct qdwhp_queue {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<qdwhp::Request*> pending;
  std::unordered_map<uint64_t, std::unique_ptr<qdwhp::Request>> all;
  std::vector<std::thread> workers;
  std::unique_ptr<qdwhp::Pool> pool;
  char* base = nullptr;
  size_t budget = 0;
  bool owns_base = false;
  bool stopping = false;
  uint64_t next_id = 1;
  int device = 0;
};

namespace qdwhp {

namespace {

void worker_loop(qdwhp_queue* q) {
  cudaSetDevice(q->device);
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
  for (;;) {
    Request* r = nullptr;
    size_t off = 0;
    {
      std::unique_lock<std::mutex> lk(q->mu);
      for (;;) {
        for (auto it = q->pending.begin(); it != q->pending.end(); ++it) {
          if (q->pool->alloc((*it)->ws_bytes, &off)) {
            r = *it;
            q->pending.erase(it);
            break;
          }
        }
        if (r != nullptr || (q->stopping && q->pending.empty())) break;
        q->cv_work.wait(lk);
      }
    }
    if (r == nullptr) break;
    r->t_start = now_s();
    qdwhp_status s = QDWHP_ERR_CUDA;
    if (st != nullptr && cudaStreamWaitEvent(st, r->ready, 0) == cudaSuccess) {
      void* ws = q->base + off;
      if (r->svd)
        s = qdwhp_svd(r->A, r->m, r->n, r->lda, r->k, &r->opts, r->vals, r->U, r->ldu, r->V, r->ldv, ws, r->ws_bytes,
                      &r->info, st);
      else
        s = qdwhp_eig(r->A, r->n, r->lda, &r->opts, r->vals, r->V, r->ldv, ws, r->ws_bytes, &r->info, st);
      if (cudaStreamSynchronize(st) != cudaSuccess && s == QDWHP_OK) s = QDWHP_ERR_CUDA;
    }
    {
      std::lock_guard<std::mutex> lk(q->mu);
      q->pool->release(off);
      r->status = s;
      r->t_done = now_s();
      r->done = true;
    }
    q->cv_done.notify_all();
    q->cv_work.notify_all();
  }
  if (st != nullptr) cudaStreamDestroy(st);
}

qdwhp_status submit(qdwhp_queue* q, std::unique_ptr<Request> r, void* caller_stream, uint64_t* req_id) {
  if (r->ws_bytes == 0) return QDWHP_ERR_ARG;
  if (r->ws_bytes + 256 > q->budget) return QDWHP_ERR_QUEUE_FULL;
  QDWHP_CUDA_TRY(cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming));
  QDWHP_CUDA_TRY(cudaEventRecord(r->ready, (cudaStream_t)caller_stream));
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(q->mu);
    r->id = q->next_id++;
    *req_id = r->id;
    q->pending.push_back(r.get());
    q->all[r->id] = std::move(r);
  }
  q->cv_work.notify_one();
  return QDWHP_OK;
}

}  // namespace

}  // namespace qdwhp

using namespace qdwhp;

extern "C" {

QDWHP_API qdwhp_status qdwhp_queue_create(size_t hbm_budget_bytes, int32_t max_slots, void* stream,
                                          qdwhp_queue** out) {
  (void)stream;
  if (out == nullptr || max_slots < 1 || max_slots > 256 || hbm_budget_bytes < (1u << 20)) return QDWHP_ERR_ARG;
  *out = nullptr;
  auto q = std::make_unique<qdwhp_queue>();
  QDWHP_CUDA_TRY(cudaGetDevice(&q->device));
  void* p = nullptr;
  if (cudaMalloc(&p, hbm_budget_bytes) != cudaSuccess) {
    cudaGetLastError();
    return QDWHP_ERR_NOMEM;
  }
  q->base = static_cast<char*>(p);
  q->owns_base = true;
  q->budget = hbm_budget_bytes;
  q->pool = std::make_unique<Pool>(hbm_budget_bytes);
  for (int i = 0; i < max_slots; ++i) q->workers.emplace_back(worker_loop, q.get());
  *out = q.release();
  return QDWHP_OK;
}

QDWHP_API qdwhp_status qdwhp_submit_eig(qdwhp_queue* q, const double* A, int64_t n, int64_t lda, const qdwhp_opts* opts,
                                        double* lambda, double* V, int64_t ldv, void* stream, uint64_t* req_id) {
  if (!q || !A || !opts || !lambda || !V || !req_id || n < 1 || lda < n || ldv < n) return QDWHP_ERR_ARG;
  auto r = std::make_unique<Request>();
  r->A = A;
  r->n = n;
  r->lda = lda;
  r->opts = *opts;
  r->vals = lambda;
  r->V = V;
  r->ldv = ldv;
  r->ws_bytes = qdwhp_eig_workspace_bytes(n, opts);
  return submit(q, std::move(r), stream, req_id);
}

QDWHP_API qdwhp_status qdwhp_submit_svd(qdwhp_queue* q, const double* A, int64_t m, int64_t n, int64_t lda, int64_t k,
                                        const qdwhp_opts* opts, double* sigma, double* U, int64_t ldu, double* V,
                                        int64_t ldv, void* stream, uint64_t* req_id) {
  if (!q || !A || !opts || !sigma || !U || !V || !req_id || m < 1 || n < 1 || lda < m || ldu < m || ldv < n)
    return QDWHP_ERR_ARG;
  auto r = std::make_unique<Request>();
  r->svd = true;
  r->A = A;
  r->m = m;
  r->n = n;
  r->lda = lda;
  r->k = k;
  r->opts = *opts;
  r->vals = sigma;
  r->U = U;
  r->ldu = ldu;
  r->V = V;
  r->ldv = ldv;
  r->ws_bytes = qdwhp_svd_workspace_bytes(m, n, opts);
  return submit(q, std::move(r), stream, req_id);
}

QDWHP_API qdwhp_status qdwhp_poll(qdwhp_queue* q, uint64_t req_id, qdwhp_info* info) {
  if (!q) return QDWHP_ERR_ARG;
  std::lock_guard<std::mutex> lk(q->mu);
  auto it = q->all.find(req_id);
  if (it == q->all.end()) return QDWHP_ERR_ARG;
  if (!it->second->done) return QDWHP_PENDING;
  if (info) *info = it->second->info;
  return it->second->status;
}

QDWHP_API qdwhp_status qdwhp_wait(qdwhp_queue* q, uint64_t req_id, int32_t timeout_ms, qdwhp_info* info) {
  if (!q) return QDWHP_ERR_ARG;
  std::unique_lock<std::mutex> lk(q->mu);
  auto it = q->all.find(req_id);
  if (it == q->all.end()) return QDWHP_ERR_ARG;
  Request* r = it->second.get();
  const bool ok = q->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                      [r] { return r->done; });
  if (!ok) return QDWHP_ERR_TIMEOUT;
  if (info) *info = r->info;
  return r->status;
}

QDWHP_API qdwhp_status qdwhp_request_times(qdwhp_queue* q, uint64_t req_id, double* t_submit, double* t_start,
                                           double* t_done) {
  if (!q) return QDWHP_ERR_ARG;
  std::lock_guard<std::mutex> lk(q->mu);
  auto it = q->all.find(req_id);
  if (it == q->all.end()) return QDWHP_ERR_ARG;
  if (t_submit) *t_submit = it->second->t_submit;
  if (t_start) *t_start = it->second->t_start;
  if (t_done) *t_done = it->second->t_done;
  return it->second->done ? QDWHP_OK : QDWHP_PENDING;
}

QDWHP_API qdwhp_status qdwhp_release(qdwhp_queue* q, uint64_t req_id) {
  if (!q) return QDWHP_ERR_ARG;
  std::lock_guard<std::mutex> lk(q->mu);
  auto it = q->all.find(req_id);
  if (it == q->all.end()) return QDWHP_ERR_ARG;
  if (!it->second->done) return QDWHP_PENDING;
  if (it->second->ready) cudaEventDestroy(it->second->ready);
  q->all.erase(it);
  return QDWHP_OK;
}

QDWHP_API qdwhp_status qdwhp_queue_destroy(qdwhp_queue* q) {
  if (!q) return QDWHP_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(q->mu);
    q->stopping = true;
  }
  q->cv_work.notify_all();
  for (auto& t : q->workers) t.join();
  for (auto& kv : q->all)
    if (kv.second->ready) cudaEventDestroy(kv.second->ready);
  if (q->owns_base && q->base) cudaFree(q->base);
  delete q;
  return QDWHP_OK;
}

QDWHP_API qdwhp_status qdwhp_eig_batched(int64_t count, const double* const* A, const int64_t* n, const int64_t* lda,
                                         const qdwhp_opts* opts, double* const* lambda, double* const* V,
                                         const int64_t* ldv, int32_t concurrency, qdwhp_status* statuses,
                                         qdwhp_info* infos, void* stream) {
  if (count < 0 || (count > 0 && (!A || !n || !lda || !opts || !lambda || !V || !ldv || !statuses))) return QDWHP_ERR_ARG;
  if (count == 0) return QDWHP_OK;
  if (concurrency < 1) concurrency = 8;
  // Largest first (longest-processing-time order), budget = the `concurrency` largest workspaces.
  std::vector<int64_t> order(count);
  for (int64_t i = 0; i < count; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return n[a] > n[b]; });
  size_t budget = 0;
  for (int64_t i = 0; i < count && i < concurrency; ++i)
    budget += ((qdwhp_eig_workspace_bytes(n[order[i]], opts) + 255) & ~size_t(255)) + 256;
  budget = std::max<size_t>(budget, 1u << 20);
  qdwhp_queue* q = nullptr;
  QDWHP_TRY(qdwhp_queue_create(budget, concurrency, stream, &q));
  std::vector<uint64_t> ids(count, 0);
  qdwhp_status first_err = QDWHP_OK;
  for (int64_t j = 0; j < count; ++j) {
    const int64_t i = order[j];
    statuses[i] = qdwhp_submit_eig(q, A[i], n[i], lda[i], opts, lambda[i], V[i], ldv[i], stream, &ids[i]);
  }
  for (int64_t i = 0; i < count; ++i) {
    if (statuses[i] != QDWHP_OK) {
      if (first_err == QDWHP_OK) first_err = statuses[i];
      continue;
    }
    qdwhp_info inf;
    // Waits are bounded: one hour in one-minute slices, then the request counts as timed out.
    qdwhp_status s = QDWHP_ERR_TIMEOUT;
    for (int slice = 0; slice < 60 && s == QDWHP_ERR_TIMEOUT; ++slice) s = qdwhp_wait(q, ids[i], 60000, &inf);
    statuses[i] = s;
    if (infos) infos[i] = inf;
    if (s != QDWHP_OK && first_err == QDWHP_OK) first_err = s;
  }
  qdwhp_queue_destroy(q);
  return first_err;
}

}  // extern "C"
