// Serving runtime: a stream of independent fixed-precision farPCA requests on
// one GPU (arxiv 2506.03859, Alg. 1 / Alg. 2 per request).
//
// Requests are queued on submission and admitted in arrival order by the
// policy of serve_policy.h: a worker slot must be free and the request's
// workspace (lra_workspace_bytes) must fit in the device-memory budget beside
// the running requests.  Each worker thread owns a CUDA stream; an admitted
// request gets a context on that stream whose memory comes from the device's
// stream-ordered pool (LRA_FLAG_POOL), so creating and freeing contexts never
// synchronises the device under the other workers, and the block steps of the
// running requests interleave on the GPU.  A request's Omega is drawn from its
// own Philox key, so its result does not depend on what runs beside it.
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.cuh"
#include "serve_policy.h"

namespace {

struct Item {
  lra_request req;
  double t_submit;
};

}  // namespace

struct lra_server {
  lra_server_params prm{};
  int dev = 0;
  lra::Admission<Item>* adm = nullptr;  // guarded by mu
  std::mutex mu;
  std::condition_variable cv_work;  // workers: admissible work or stop
  std::condition_variable cv_done;  // pollers: a completion, or nothing pending
  std::deque<lra_completion> done;
  std::unordered_map<lra_ctx*, int64_t> kept;  // contexts kept for the caller -> bytes
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  int64_t pending = 0;
  bool stop = false;
  std::chrono::steady_clock::time_point t0;
  cudaMemPool_t mempool = nullptr;
  uint64_t old_threshold = 0;
};

namespace {

double clock_of(const lra_server* s) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

lra_completion run_one(lra_server* s, const Item& it, double t_admit, cudaStream_t st) {
  lra_completion c;
  memset(&c, 0, sizeof c);
  c.id = it.req.id;
  c.t_submit = it.t_submit;
  c.t_admit = t_admit;
  lra_params p = it.req.params;
  p.flags |= s->prm.flags | LRA_FLAG_POOL;
  lra_ctx* ctx = nullptr;
  lra_status st_ = lra_create(&ctx, it.req.A.m, it.req.A.n, &p, st);
  c.t_start = clock_of(s);
  if (st_ == LRA_OK) {
    st_ = lra_farpca_run(ctx, &it.req.A);
    lra_result_t r;
    lra_result(ctx, &r);
    c.rank = r.rank;
    c.rel_err = r.rel_err;
    c.bytes = lra_device_bytes(ctx);
  }
  c.status = st_;
  c.t_done = clock_of(s);
  if (ctx && it.req.keep && st_ >= 0) {
    c.ctx = ctx;
  } else if (ctx) {
    lra_destroy(ctx);
  }
  return c;
}

void worker(lra_server* s, int slot) {
  cudaSetDevice(s->dev);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    Item it;
    int64_t bytes = 0;
    while (!s->adm->admit(&it, &bytes)) {
      if (s->stop && s->adm->waiting() == 0) return;
      s->cv_work.wait(lk);
    }
    const double t_admit = clock_of(s);
    lk.unlock();
    lra_completion c = run_one(s, it, t_admit, s->streams[slot]);
    lk.lock();
    if (c.ctx) {
      s->kept[c.ctx] = bytes;
      s->adm->finish(0);  // the slot is free; the bytes stay with the kept context
    } else {
      s->adm->finish(bytes);
    }
    s->done.push_back(c);
    --s->pending;
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

}  // namespace

extern "C" {

lra_status lra_server_create(lra_server** out, const lra_server_params* params) {
  if (!out || !params) return LRA_ERR_INVALID_ARG;
  *out = nullptr;
  if (params->slots < 1 || params->slots > 64 || params->hbm_budget < 0)
    return LRA_ERR_INVALID_ARG;
  lra_server* s = new lra_server();
  s->prm = *params;
  s->t0 = std::chrono::steady_clock::now();
  if (cudaGetDevice(&s->dev) != cudaSuccess) {
    delete s;
    return LRA_ERR_CUDA;
  }
  int64_t budget = params->hbm_budget;
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete s;
      return LRA_ERR_CUDA;
    }
    budget = (int64_t)(0.9 * (double)fr);
  }
  s->adm = new lra::Admission<Item>(budget, params->slots);
  // kernel attributes once, before the workers run; freed pool memory stays
  // in the pool up to the budget instead of going back to the driver
  cudaError_t e = lra::gather_prepare();
  if (e == cudaSuccess) e = lra::oz_prepare();
  if (e == cudaSuccess) e = cudaDeviceGetDefaultMemPool(&s->mempool, s->dev);
  if (e == cudaSuccess)
    e = cudaMemPoolGetAttribute(s->mempool, cudaMemPoolAttrReleaseThreshold, &s->old_threshold);
  if (e == cudaSuccess) {
    uint64_t thr = (uint64_t)budget;
    e = cudaMemPoolSetAttribute(s->mempool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  for (int i = 0; i < params->slots && e == cudaSuccess; ++i) {
    cudaStream_t st = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) s->streams.push_back(st);
  }
  if (e != cudaSuccess) {
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    delete s->adm;
    delete s;
    cudaGetLastError();
    return LRA_ERR_CUDA;
  }
  for (int i = 0; i < params->slots; ++i) s->workers.emplace_back(worker, s, i);
  *out = s;
  return LRA_OK;
}

lra_status lra_server_submit(lra_server* s, const lra_request* req) {
  if (!s || !req) return LRA_ERR_INVALID_ARG;
  const lra_matrix& A = req->A;
  if (!A.data || A.m < 1 || A.n < 1 || A.lda < A.m || (A.dtype != LRA_F64 && A.dtype != LRA_F32))
    return LRA_ERR_INVALID_ARG;
  lra_params p = req->params;
  p.flags |= s->prm.flags | LRA_FLAG_POOL;
  const int64_t bytes = lra_workspace_bytes(A.m, A.n, &p);
  if (bytes < 0) return (lra_status)bytes;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return LRA_ERR_INVALID_ARG;
  if (!s->adm->submit(Item{*req, clock_of(s)}, bytes)) return LRA_ERR_UNSUPPORTED;
  ++s->pending;
  s->cv_work.notify_all();
  return LRA_OK;
}

int64_t lra_server_poll(lra_server* s, lra_completion* out, int64_t max, int32_t wait) {
  if (!s || (!out && max > 0) || max < 0) return LRA_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  if (wait) s->cv_done.wait(lk, [&] { return !s->done.empty() || s->pending == 0; });
  int64_t k = 0;
  while (k < max && !s->done.empty()) {
    out[k++] = s->done.front();
    s->done.pop_front();
  }
  return k;
}

int64_t lra_server_pending(const lra_server* s) {
  if (!s) return -1;
  std::lock_guard<std::mutex> lk(const_cast<lra_server*>(s)->mu);
  return s->pending;
}

lra_status lra_server_release(lra_server* s, lra_ctx* ctx) {
  if (!s || !ctx) return LRA_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->kept.find(ctx);
    if (it == s->kept.end()) return LRA_ERR_INVALID_ARG;
    s->adm->free_bytes(it->second);
    s->kept.erase(it);
  }
  lra_destroy(ctx);
  s->cv_work.notify_all();
  return LRA_OK;
}

double lra_server_clock(const lra_server* s) { return s ? clock_of(s) : 0.0; }

void lra_server_destroy(lra_server* s) {
  if (!s) return;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->pending == 0; });
    s->stop = true;
    s->cv_work.notify_all();
  }
  for (auto& t : s->workers) t.join();
  for (auto& kv : s->kept) lra_destroy(kv.first);
  for (cudaStream_t st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  if (s->mempool)
    cudaMemPoolSetAttribute(s->mempool, cudaMemPoolAttrReleaseThreshold, &s->old_threshold);
  delete s->adm;
  delete s;
}

}  // extern "C"
