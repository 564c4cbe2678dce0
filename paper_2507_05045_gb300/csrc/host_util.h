// Host helpers shared by the solver translation units: a stream-ordered
// device allocator that frees everything it handed out, the CUDA error
// check that maps to msp_status codes, per-launch event timing and NVTX
// ranges over the stages of a solve.
#pragma once

#include <algorithm>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "host_internal.h"

namespace msp {

struct DevAlloc {
  cudaStream_t s;
  std::vector<void *> ptrs;
  size_t bytes = 0, peak = 0;
  explicit DevAlloc(cudaStream_t st) : s(st) {}
  template <typename T>
  cudaError_t get(T **p, size_t count) {
    void *q = nullptr;
    const size_t b = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMallocAsync(&q, b, s);
    if (e != cudaSuccess) return e;
    ptrs.push_back(q);
    bytes += b;
    peak = std::max(peak, bytes);
    *p = static_cast<T *>(q);
    return cudaSuccess;
  }
  void free1(void *q, size_t b) {
    for (auto &x : ptrs)
      if (x == q) {
        cudaFreeAsync(q, s);
        x = nullptr;
        bytes -= b;
        return;
      }
  }
  void release() {
    for (void *q : ptrs)
      if (q) cudaFreeAsync(q, s);
    ptrs.clear();
    bytes = 0;
  }
  ~DevAlloc() { release(); }
};

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      return fail(e_ == cudaErrorMemoryAllocation ? MSP_ENOMEM : MSP_ECUDA,           \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                \
    }                                                                                 \
  } while (0)

// Per-launch CUDA-event timing (only when the instance has profiling on)
// and launch counting (always).
struct Prof {
  bool on = false;
  cudaStream_t s = nullptr;
  msp_stats *st = nullptr;
  struct Item {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Item> pending;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  cudaEvent_t a_ = nullptr;
  void begin() {
    if (!on) return;
    a_ = get();
    cudaEventRecord(a_, s);
  }
  void end(int kind, int kernels, uint64_t bytes) {
    st->kernel_launches += kernels;
    if (!on) return;
    cudaEvent_t b = get();
    cudaEventRecord(b, s);
    pending.push_back({kind, a_, b});
    st->kernel_count[kind] += kernels;
    st->kernel_bytes[kind] += bytes;
  }
  // call after the stream reached the recorded events
  void flush() {
    for (auto &it : pending) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, it.a, it.b) == cudaSuccess) st->kernel_ms[it.kind] += ms;
      pool.push_back(it.a);
      pool.push_back(it.b);
    }
    pending.clear();
  }
  ~Prof() {
    for (auto &it : pending) {
      cudaEventDestroy(it.a);
      cudaEventDestroy(it.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

// A small ring of events (timing off) that bounds how many launches a
// cancelable solve keeps queued: record after launch i, wait before launch
// i + size.
struct EventRing {
  std::vector<cudaEvent_t> ev;
  cudaError_t status = cudaSuccess;  // the first failed event creation, if any
  explicit EventRing(uint32_t n) : ev(n, nullptr) {
    for (auto &e : ev) {
      const cudaError_t r = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
      if (r != cudaSuccess && status == cudaSuccess) status = r;
    }
  }
  ~EventRing() {
    for (auto e : ev)
      if (e) cudaEventDestroy(e);
  }
  EventRing(const EventRing &) = delete;
  EventRing &operator=(const EventRing &) = delete;
  cudaError_t record(uint32_t i, cudaStream_t s) { return cudaEventRecord(ev[i], s); }
  cudaError_t wait(uint32_t i) { return cudaEventSynchronize(ev[i]); }
};

// NVTX range over a host stage of a solve (header-only NVTX3: with no
// profiler attached a range costs a function call that does nothing).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { end(); }
  void end() {  // close the range before the end of the scope
    if (open_) nvtxRangePop();
    open_ = false;
  }
  bool open_ = true;
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

#define LAUNCH(kind, kernels, bytes, call) \
  do {                                     \
    prof.begin();                          \
    CK(call);                              \
    prof.end(kind, kernels, bytes);        \
  } while (0)


}  // namespace msp
