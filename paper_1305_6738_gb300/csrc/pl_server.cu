// pl_server.cu -- continuous-batching engine for goodness-of-fit requests.
//
// Each request is a data set; the engine fits alpha-hat (Eq. 2), computes D
// (Eq. 3) and the parametric-bootstrap p-value with B replicates at alpha-hat
// (the paper's bespoke cutoff, Section 4).  Worker threads each own a
// library context and a CUDA stream, so the requests they hold run on the
// GPU at the same time; a request is admitted, in arrival order, when a
// worker is free and its estimated device workspace fits beside the
// workspaces of the requests already running (the device budget).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "pl.h"
#include "pl_kernels.cuh"

namespace pl {
size_t ctx_bootstrap_bytes(pl_ctx *ctx, int64_t n, uint64_t xmin, int64_t B);
uint64_t ctx_launches(const pl_ctx *ctx);
}  // namespace pl

namespace {

using clock_type = std::chrono::steady_clock;

struct Request {
  uint64_t id;
  std::vector<int32_t> data;
  uint64_t xmin;
  double submit_s;
  size_t bytes;
};

struct Worker {
  pl_ctx *ctx = nullptr;
  cudaStream_t stream = nullptr;
  int32_t *x_dev = nullptr;
  size_t x_cap = 0;
  int32_t *x_pinned = nullptr;
  std::thread thread;
};

}  // namespace

struct pl_server {
  int device = 0;
  pl_precision prec = PL_FP32_BULK;
  uint64_t seed = 1;
  int64_t B = 2500;
  size_t budget = 0;
  size_t reserved = 0;
  clock_type::time_point t0;
  pl_ctx *sizer = nullptr;  // plans request sizes on the host only (never launches)
  std::mutex sizer_mu;
  std::vector<Worker> workers;
  std::deque<Request> queue;
  std::vector<pl_result> done;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stopping = false;
  int busy = 0;
  uint64_t launches = 0;  // kernels launched by finished requests

  double now() const { return std::chrono::duration<double>(clock_type::now() - t0).count(); }
};

namespace {

void worker_loop(pl_server *srv, Worker *w) {
  cudaSetDevice(srv->device);
  for (;;) {
    Request req;
    {
      std::unique_lock<std::mutex> lock(srv->mu);
      // admission: the oldest request, once its workspace fits the budget
      srv->cv_work.wait(lock, [&] {
        return srv->stopping ||
               (!srv->queue.empty() && srv->reserved + srv->queue.front().bytes <= srv->budget);
      });
      if (srv->stopping) return;  // queued requests are dropped
      req = std::move(srv->queue.front());
      srv->queue.pop_front();
      srv->reserved += req.bytes;
      ++srv->busy;
    }
    pl_result res{};
    res.request_id = req.id;
    res.n = (int64_t)req.data.size();
    res.submit_s = req.submit_s;
    res.start_s = srv->now();
    pl_status st = PL_OK;
    const uint64_t l0 = pl::ctx_launches(w->ctx);
    const size_t nbytes = req.data.size() * sizeof(int32_t);
    if (w->x_cap < nbytes) {
      if (w->x_dev) cudaFree(w->x_dev);
      if (w->x_pinned) cudaFreeHost(w->x_pinned);
      w->x_dev = nullptr;
      w->x_pinned = nullptr;
      w->x_cap = 0;
      if (cudaMalloc(&w->x_dev, nbytes) != cudaSuccess || cudaMallocHost(&w->x_pinned, nbytes) != cudaSuccess)
        st = PL_ENOMEM;
      else
        w->x_cap = nbytes;
    }
    if (st == PL_OK) {
      std::memcpy(w->x_pinned, req.data.data(), nbytes);
      if (cudaMemcpyAsync(w->x_dev, w->x_pinned, nbytes, cudaMemcpyHostToDevice, w->stream) != cudaSuccess)
        st = PL_ECUDA;
    }
    if (st == PL_OK)
      st = pl_bootstrap_pvalue(w->ctx, w->x_dev, (int64_t)req.data.size(), req.xmin, srv->B, srv->seed,
                               req.id, srv->prec, &res.alpha_hat, &res.D, &res.p, w->stream);
    res.status = st;
    res.done_s = srv->now();
    {
      std::lock_guard<std::mutex> lock(srv->mu);
      srv->reserved -= req.bytes;
      --srv->busy;
      srv->launches += pl::ctx_launches(w->ctx) - l0;
      srv->done.push_back(res);
    }
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();
  }
}

}  // namespace

extern "C" {

pl_status pl_server_create(pl_server **out, int device, size_t mem_budget_bytes, int workers,
                           pl_precision prec, uint64_t seed, int64_t B) {
  if (!out || workers < 1 || workers > 64 || B < 1 || (prec != PL_FP64 && prec != PL_FP32_BULK))
    return PL_EINVAL;
  *out = nullptr;
  pl_server *srv = new pl_server();
  srv->device = device;
  srv->prec = prec;
  srv->seed = seed;
  srv->B = B;
  srv->budget = mem_budget_bytes ? mem_budget_bytes : (size_t)40 << 30;
  srv->t0 = clock_type::now();
  srv->workers.resize(workers);
  if (pl_status st = pl_create(&srv->sizer, device, srv->budget)) {
    delete srv;
    return st;
  }
  for (Worker &w : srv->workers) {
    pl_status st = pl_create(&w.ctx, device, srv->budget);
    if (st == PL_OK && cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking) != cudaSuccess) st = PL_ECUDA;
    if (st != PL_OK) {
      for (Worker &v : srv->workers) {
        if (v.stream) cudaStreamDestroy(v.stream);
        if (v.ctx) pl_destroy(v.ctx);
      }
      pl_destroy(srv->sizer);
      delete srv;
      return st;
    }
  }
  for (Worker &w : srv->workers) w.thread = std::thread(worker_loop, srv, &w);
  *out = srv;
  return PL_OK;
}

pl_status pl_server_submit(pl_server *srv, uint64_t request_id, const int32_t *x_host, int64_t n, uint64_t xmin) {
  if (!srv || !x_host || n < 1 || xmin < 1 || request_id >= (1ull << 32)) return PL_EINVAL;
  Request req;
  req.id = request_id;
  req.data.assign(x_host, x_host + n);
  req.xmin = xmin;
  req.submit_s = srv->now();
  {
    std::lock_guard<std::mutex> lock(srv->sizer_mu);
    req.bytes = pl::ctx_bootstrap_bytes(srv->sizer, n, xmin, srv->B);
  }
  if (req.bytes > srv->budget) {  // can never be admitted: fails at once
    pl_result res{};
    res.request_id = req.id;
    res.status = PL_ENOMEM;
    res.n = n;
    res.submit_s = res.start_s = res.done_s = req.submit_s;
    res.alpha_hat = res.D = res.p = std::nan("");
    {
      std::lock_guard<std::mutex> lock(srv->mu);
      srv->done.push_back(res);
    }
    srv->cv_done.notify_all();
    return PL_OK;
  }
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    srv->queue.push_back(std::move(req));
  }
  srv->cv_work.notify_one();
  return PL_OK;
}

int pl_server_poll(pl_server *srv, pl_result *out, int max_results, double wait_s) {
  if (!srv || !out || max_results < 1) return 0;
  std::unique_lock<std::mutex> lock(srv->mu);
  if (srv->done.empty() && wait_s > 0.0)
    srv->cv_done.wait_for(lock, std::chrono::duration<double>(wait_s), [&] { return !srv->done.empty(); });
  const int k = (int)std::min<size_t>((size_t)max_results, srv->done.size());
  for (int i = 0; i < k; ++i) out[i] = srv->done[i];
  srv->done.erase(srv->done.begin(), srv->done.begin() + k);
  return k;
}

double pl_server_now(const pl_server *srv) { return srv ? srv->now() : 0.0; }

pl_status pl_server_load(pl_server *srv, int *queued, int *running, size_t *reserved_bytes,
                         uint64_t *launches) {
  if (!srv) return PL_EINVAL;
  std::lock_guard<std::mutex> lock(srv->mu);
  if (queued) *queued = (int)srv->queue.size();
  if (running) *running = srv->busy;
  if (reserved_bytes) *reserved_bytes = srv->reserved;
  if (launches) *launches = srv->launches;
  return PL_OK;
}

void pl_server_destroy(pl_server *srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    srv->stopping = true;
  }
  srv->cv_work.notify_all();
  for (Worker &w : srv->workers)
    if (w.thread.joinable()) w.thread.join();
  for (Worker &w : srv->workers) {
    if (w.stream) cudaStreamDestroy(w.stream);
    if (w.x_dev) cudaFree(w.x_dev);
    if (w.x_pinned) cudaFreeHost(w.x_pinned);
    if (w.ctx) pl_destroy(w.ctx);
  }
  pl_destroy(srv->sizer);
  delete srv;
}

}  // extern "C"
