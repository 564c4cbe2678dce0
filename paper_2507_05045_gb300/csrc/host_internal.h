// Host-side declarations shared by solver.cu and server.cu.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/msp.h"

struct msp_instance {
  int m = 0, n = 0;
  const volatile int *cancel = nullptr;  // non-null: checked between passes
  std::vector<int32_t> A, d;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t budget = 0;
  msp_stats stats{};
  int device = 0;
  bool profiling = false;
  bool force_exact = false;
};

namespace msp {
// Sets the calling thread's error text and returns `code`.
int fail(int code, const std::string &msg);
// msp_solve_all without the argument checks of the C entry point.
int solve_instance(msp_instance *inst, uint64_t **masks, size_t *count, int *words);
// Device bytes of the quarter lists plus one residue pass (capped at cap).
size_t footprint_estimate(int m, int n, size_t cap);
}  // namespace msp
