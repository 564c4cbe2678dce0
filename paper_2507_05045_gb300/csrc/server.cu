// Serving loop of libmsp: msp_server_create / msp_submit / msp_poll.
//
// Requests of mixed (m, n) wait in a queue in arrival order.  A request is
// admitted as soon as a worker slot is free and its device footprint
// (footprint_estimate) fits in what the budget has left; a large request
// (more than about 2^32 half-pair records) also waits until no other large
// one is running;
// the footprint also caps that request's pass buffers, so admitted requests
// never exceed the budget together.  Each worker runs its request's residue
// passes on its own CUDA stream, so the passes of all admitted requests are
// interleaved on the device, and requests that arrive while others run are
// admitted as slots and memory free up (continuous batching).  Small
// requests run on high-priority streams, so they overtake the kernels of
// large ones at the next launch boundary.
#include "host_internal.h"

#include <atomic>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

namespace {

enum ReqState { kQueued, kRunning, kDone, kFailed, kCanceled };

struct Request {
  uint64_t id = 0;
  int m = 0, n = 0;
  std::vector<int32_t> A, d;
  size_t footprint = 0;
  bool urgent = false;  // small request: runs on the worker's high-priority stream
  ReqState state = kQueued;
  int rc = MSP_OK;
  std::string err;
  uint64_t *masks = nullptr;
  size_t count = 0;
  int words = 1;
  volatile int cancel = 0;
};

}  // namespace

struct msp_server {
  size_t budget = 0;
  size_t in_use = 0;
  int max_inflight = 1;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Request *> reqs;
  std::vector<std::thread> workers;
  bool stop = false;
  uint64_t next_id = 1;
  int large_running = 0;  // admitted requests that are not small
};

namespace {

void worker_loop(msp_server *srv) {
  cudaSetDevice(srv->device);
  // Two streams: small requests on the high-priority one, so that their
  // kernels take SMs ahead of the (bounded, ~15 ms) launches of large
  // requests running on the other workers' low-priority streams.
  int least = 0, greatest = 0;
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  cudaStream_t stream = nullptr, urgent_stream = nullptr;
  cudaStreamCreateWithPriority(&stream, cudaStreamNonBlocking, least);
  cudaStreamCreateWithPriority(&urgent_stream, cudaStreamNonBlocking, greatest);
  for (;;) {
    Request *rq = nullptr;
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      for (;;) {
        if (srv->stop) {
          lk.unlock();
          if (stream) cudaStreamDestroy(stream);
          if (urgent_stream) cudaStreamDestroy(urgent_stream);
          return;
        }
        // Admission in arrival order, by size: a small request runs as soon
        // as a worker and its footprint are free; a large one (whose kernels
        // fill the GPU by themselves) waits until no other large request is
        // running, so large requests run one after another at full speed
        // while small ones pass them.
        while (!srv->queue.empty()) {
          auto it = srv->reqs.find(srv->queue.front());
          if (it == srv->reqs.end() || it->second->state != kQueued) {
            srv->queue.pop_front();
            continue;
          }
          break;
        }
        bool large_waits = srv->large_running > 0;
        for (auto qi = srv->queue.begin(); qi != srv->queue.end(); ++qi) {
          auto it = srv->reqs.find(*qi);
          if (it == srv->reqs.end() || it->second->state != kQueued) continue;
          Request *cand = it->second;
          if (!cand->urgent && large_waits) continue;
          if (srv->in_use == 0 || srv->in_use + cand->footprint <= srv->budget) {
            srv->queue.erase(qi);
            rq = cand;
            rq->state = kRunning;
            srv->in_use += rq->footprint;
            if (!rq->urgent) ++srv->large_running;
            break;
          }
          // the oldest large request keeps its turn until memory frees up
          if (!cand->urgent) large_waits = true;
        }
        if (rq) break;
        srv->cv.wait(lk);
      }
    }
    msp_instance inst;
    inst.m = rq->m;
    inst.n = rq->n;
    inst.A = rq->A;
    inst.d = rq->d;
    inst.stream = rq->urgent ? urgent_stream : stream;
    inst.own_stream = false;
    inst.budget = rq->footprint;
    inst.device = srv->device;
    inst.cancel = &rq->cancel;
    uint64_t *masks = nullptr;
    size_t count = 0;
    int words = 1;
    const int rc = msp::solve_instance(&inst, &masks, &count, &words);
    const std::string err = rc == MSP_OK ? std::string() : std::string(msp_last_error());
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      srv->in_use -= rq->footprint;
      if (!rq->urgent) --srv->large_running;
      rq->rc = rc;
      rq->err = err;
      rq->masks = masks;
      rq->count = count;
      rq->words = words;
      rq->state = rc == MSP_OK ? kDone : (rc == MSP_ECANCELED ? kCanceled : kFailed);
    }
    srv->cv.notify_all();
  }
}

}  // namespace

extern "C" {

int msp_server_create(size_t hbm_budget_bytes, int max_inflight, msp_server **out) {
  if (!out) return msp::fail(MSP_EINVAL, "out must be non-null");
  *out = nullptr;
  if (max_inflight < 1 || max_inflight > 64) return msp::fail(MSP_ERANGE, "max_inflight must lie in [1, 64]");
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1)
    return msp::fail(MSP_ECUDA, "no CUDA device available");
  auto *srv = new (std::nothrow) msp_server();
  if (!srv) return msp::fail(MSP_ENOMEM, "host allocation failed");
  cudaGetDevice(&srv->device);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    delete srv;
    return msp::fail(MSP_ECUDA, "cudaMemGetInfo failed");
  }
  srv->budget = hbm_budget_bytes ? hbm_budget_bytes : static_cast<size_t>(0.8 * free_b);
  srv->max_inflight = max_inflight;
  for (int k = 0; k < max_inflight; ++k) srv->workers.emplace_back(worker_loop, srv);
  *out = srv;
  return MSP_OK;
}

int msp_submit(msp_server *srv, const int32_t *A, const int32_t *d, int m, int n, uint64_t *req_id) {
  if (!srv || !A || !d || !req_id) return msp::fail(MSP_EINVAL, "null argument");
  // the same checks as msp_create
  if (m < 1 || m > 16) return msp::fail(MSP_ERANGE, "m must lie in [1, 16]");
  if (n < 1 || n > 100) return msp::fail(MSP_ERANGE, "n must lie in [1, 100]");
  for (int i = 0; i < m; ++i) {
    if (d[i] < 0) return msp::fail(MSP_EINVAL, "d has a negative entry");
    int64_t s = 0;
    for (int j = 0; j < n; ++j) {
      if (A[(size_t)i * n + j] < 0) return msp::fail(MSP_EINVAL, "A has a negative entry");
      s += A[(size_t)i * n + j];
    }
    if (s >= 65536) return msp::fail(MSP_ERANGE, "a row sum reaches 2^16");
  }
  auto *rq = new (std::nothrow) Request();
  if (!rq) return msp::fail(MSP_ENOMEM, "host allocation failed");
  rq->m = m;
  rq->n = n;
  rq->A.assign(A, A + (size_t)m * n);
  rq->d.assign(d, d + m);
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    rq->footprint = msp::footprint_estimate(m, n, srv->budget / static_cast<size_t>(srv->max_inflight));
    rq->urgent = n <= 62;  // at most about 2^32 half-pair records
    if (rq->footprint > srv->budget) {
      delete rq;
      return msp::fail(MSP_ENOMEM, "request footprint exceeds the server budget");
    }
    rq->id = srv->next_id++;
    srv->reqs[rq->id] = rq;
    srv->queue.push_back(rq->id);
    *req_id = rq->id;
  }
  srv->cv.notify_all();
  return MSP_OK;
}

int msp_poll(msp_server *srv, uint64_t req_id, uint64_t **masks, size_t *count, int *words) {
  if (!srv || !masks || !count) return msp::fail(MSP_EINVAL, "null argument");
  *masks = nullptr;
  *count = 0;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(req_id);
  if (it == srv->reqs.end()) return msp::fail(MSP_EINVAL, "unknown request id");
  Request *rq = it->second;
  if (rq->state == kQueued || rq->state == kRunning) return MSP_PENDING;
  int rc = rq->rc;
  if (rq->state == kDone) {
    *masks = rq->masks;
    *count = rq->count;
    if (words) *words = rq->words;
  } else {
    msp::fail(rc, rq->err.empty() ? "request failed" : rq->err);
  }
  srv->reqs.erase(it);
  delete rq;
  return rc;
}

int msp_cancel(msp_server *srv, uint64_t req_id) {
  if (!srv) return msp::fail(MSP_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(req_id);
  if (it == srv->reqs.end()) return msp::fail(MSP_EINVAL, "unknown request id");
  Request *rq = it->second;
  if (rq->state == kQueued) {
    rq->state = kCanceled;
    rq->rc = MSP_ECANCELED;
    rq->err = "request canceled";
  } else if (rq->state == kRunning) {
    rq->cancel = 1;
  }
  return MSP_OK;
}

void msp_server_destroy(msp_server *srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
    for (auto &kv : srv->reqs)
      if (kv.second->state == kRunning) kv.second->cancel = 1;
  }
  srv->cv.notify_all();
  for (auto &t : srv->workers) t.join();
  for (auto &kv : srv->reqs) {
    std::free(kv.second->masks);
    delete kv.second;
  }
  delete srv;
}

}  // extern "C"
