// Host-side declarations shared by solver.cu and server.cu.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/msp.h"
#include "msp_internal.cuh"

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
  int64_t part = 0, parts = 1;  // residue-class subset [part*M/parts, (part+1)*M/parts)
  int plan_B = -1, plan_D = -1, plan_inner = -1;  // plan overrides (-1 = formula)
  int direct = -1;      // direct pass: -1 auto, 0 never, 1 whenever the instance fits it
  int table_bits = -1;  // direct pass shared-table bits (-1 = default)
  bool first_only = false;  // direct pass: stop once a solution is found
  uint64_t wait_ns = msp::kDefaultWaitNs;  // streaming join: limit of each bounded wait
  int wait_check = 0;       // streaming join: each block first waits on a phase no copy completes
};

namespace msp {

// Solve plan of an (m, n) instance: quarters, residue classes, digits.
struct Plan {
  int m, n, W;
  int q[4], col0[4];
  int lgL, lgR;        // log2 |L|, |R|
  int B, t, D, Dx, S;  // D: streaming-pass digits, Dx: exact-pass digits
  uint32_t c_row[kMaxClassRows];
  uint64_t w_row[kMaxRows];
};

// Plan choices that override the formulas of make_plan (-1 = formula):
// class bits B (residue modulus 2^B), digit bits D of the streaming pass,
// inner bits (the inner quarter of each side gets B + inner bits columns).
struct PlanChoice {
  int B = -1, D = -1, inner = -1;
};
Plan make_plan(int m, int n, const PlanChoice &ch = PlanChoice());
// Argument checks shared by the entry points (MSP_OK or an error status).
int validate(const int32_t *A, const int32_t *d, int m, int n);
// K(v) and kappa(v) of a vector of row sums under a plan.
uint64_t key_of(const Plan &p, const int64_t *v);
uint32_t class_of(const Plan &p, const int64_t *v);

// Sets the calling thread's error text and returns `code`.
int fail(int code, const std::string &msg);
// msp_solve_all without the argument checks of the C entry point.
int solve_instance(msp_instance *inst, uint64_t **masks, size_t *count, int *words);
// Solve count instances of one (m, n) together on stream s (raw[k]: unsorted
// two-word masks of instance k); budget 0 = most of the free device memory.
int solve_batch_impl(const int32_t *const *A, const int32_t *const *d, int m, int n, int count,
                     std::vector<std::vector<uint64_t>> &raw, cudaStream_t s, size_t budget);
// Device bytes of the quarter lists plus one residue pass (capped at cap).
size_t footprint_estimate(int m, int n, size_t cap);

// Direct pass (direct.cu): the columns of each half are split into an outer
// quarter of at most 2^10 subsets and an inner quarter bucketed into 2^B
// residue classes of about 16 subsets, so that one block joins a class
// (about 2^13 records per side) in shared memory.
struct DirectPlan {
  bool ok;            // the instance fits the direct pass
  int m, n, W;
  int cols[2];        // columns of L (the first ceil(n/2)) and R
  int qo[2], qi[2];   // outer and inner quarter columns per side
  int col_o[2], col_i[2];
  int B, t;           // residue classes 2^B over rows 1..t
  int TB;             // shared table of 2^TB slots
};
DirectPlan make_direct_plan(int m, int n, int table_bits);
// Device bytes of a direct solve.
size_t direct_footprint(const DirectPlan &d);
constexpr int kDirectFallback = 2;            // solve_direct: use another path
constexpr uint64_t kDirectMatchCap = 1u << 23;  // matched (class, key) pairs held
struct Prof;
int solve_direct(msp_instance *inst, const DirectPlan &dp, const Plan &kp, size_t budget, Prof &prof,
                 std::vector<uint64_t> &res);
// msp_solve_batch on the direct pass (MSP_OK, kDirectFallback or an error).
int solve_batch_direct(const int32_t *const *A, const int32_t *const *d, int m, int n, int count,
                       std::vector<std::vector<uint64_t>> &raw, cudaStream_t s, size_t budget);
// Device memory a solve may use: the instance budget, else 85% of what is
// free (counting the stream-ordered pool's unused memory as free).
size_t solve_budget(const msp_instance *inst, size_t already_held);
}  // namespace msp
