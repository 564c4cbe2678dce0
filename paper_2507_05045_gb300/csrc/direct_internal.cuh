// Shared declarations of the direct pass (direct_join.cu: the class joins,
// direct_kernels.cu: list builds, verification and C1, direct.cu: host
// side).  The direct pass joins residue classes of about 2^13 records per
// side entirely in shared memory; direct_kernels.cu describes the method.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace msp {

constexpr int kDirectThreads = 512;          // threads per join block
constexpr int kOuterMax = kDirectThreads;    // outer subsets per side: one per thread of a join block
constexpr int kInnerMax = 31;                // inner quarter columns (32-bit positions)
constexpr int kGenChunk = 6;                 // Gray walk of 2^6 subsets per thread
constexpr int kVerifyPairSlots = 256;        // counters of checked pairs in verification

struct InnerGen {
  uint32_t ck[kInnerMax];  // 32-bit key of each column (row sums weighted by w_i)
  uint32_t cc[kInnerMax];  // class contribution of each column (unmasked)
  int q;                   // columns of the quarter
  int neg;                 // 1: store -K and -kappa (right inner list)
  uint32_t cmask;
};

// The inner quarter of one side of one instance of a batch: its column
// tables and its lists.
struct InnerSeg {
  InnerGen g;
  uint32_t *cnt;    // [2^B] counts, then insertion cursors
  uint32_t *ioff;   // [2^B + 1] bucket starts
  uint32_t *ikey;   // [2^q] keys in bucket order
  uint32_t *imask;  // [2^q] subset masks in bucket order
};

struct DirectSide {
  const uint32_t *okey;  // [no] outer keys (transformed on the right)
  const uint32_t *ocls;  // [no] outer classes (transformed, masked)
  const uint32_t *ikey;  // [ni] inner keys, bucketed by class
  const uint32_t *ioff;  // [M + 1] bucket starts
  int no;
};

// One instance of a direct pass (device table: one entry for a single
// solve, one per instance of a batch of the same (m, n)).
struct DirectInst {
  DirectSide side[2];
};

struct DirectPass {
  const DirectInst *inst;  // [ninst]
  uint32_t ninst;
  int no[2];              // outer subsets per side (the same for every instance)
  uint32_t class_bits;    // a match is tagged instance << class_bits | class
  uint32_t cmask;
  uint32_t c0;            // first class of the launch
  uint32_t nclass;        // classes of the launch
  uint32_t chunk;         // consecutive classes per work item
  unsigned int *work;     // work-item counter (zeroed before the launch)
  uint32_t insert_cap;    // left keys per table fill
  uint32_t *match_key;
  uint32_t *match_cls;
  unsigned long long *match_count;
  uint64_t match_cap;
  unsigned long long *records;  // records generated (both sides)
  unsigned int *error;    // a bucket or class beyond the kernel's 32-bit bounds
};

// The lists of one instance that verification reads.
struct DirectVerifyInst {
  DirectSide side[2];
  const uint32_t *imask[2];  // inner subset masks (bucketed order)
  const uint32_t *omask[2];  // outer subset masks
  const uint64_t *ovec[2];   // [no][4] packed row sums of the outer subsets
  const uint64_t *icol[2];   // [qi][4] packed column vectors of the inner quarters
  uint64_t dvec[4];          // packed right-hand side
};

struct DirectVerify {
  const DirectVerifyInst *inst;  // [ninst], indexed by a match's tag
  int qi[2];
  int col_o[2], col_i[2];    // first column of each quarter
  int W;                     // packed words in use
  uint32_t class_bits;
  uint32_t cmask;
  const uint32_t *match_key;
  const uint32_t *match_cls; // instance << class_bits | class
  uint64_t *sol;             // [sol_cap][3]: mask low word, high word, instance
  unsigned long long *sol_count;
  uint64_t sol_cap;
  unsigned long long *pairs; // [kVerifyPairSlots] candidate pairs checked (summed by the host)
  unsigned int *overflow;    // a match had more candidates than the block holds
};

// Launchers (asynchronous on s; return cudaGetLastError()).
// Counts the 2^q subsets of one inner quarter by class into cnt_or_cur
// (ikey == nullptr), or places them at the cursors cnt_or_cur.
cudaError_t launch_direct_inner(const InnerGen &g, uint32_t *cnt_or_cur, uint32_t *ikey, uint32_t *imask,
                                cudaStream_t s);
// The same for the inner quarters of every segment of a batch (all of q
// columns): counts (scatter = false) or placement.
cudaError_t launch_direct_inner_batch(const InnerSeg *segs, int nseg, int q, bool scatter, cudaStream_t s);
// Bucket starts of every segment of a batch (2^B <= 2^20): one block each.
cudaError_t launch_direct_inner_offsets(const InnerSeg *segs, int nseg, uint32_t M, cudaStream_t s);
// Class joins of a launch's classes [p.c0, p.c0 + p.nclass) of every instance.
cudaError_t launch_direct_join(int TB, const DirectPass &p, cudaStream_t s);
// Recovery and all-row verification of nmatch matches, one block each.
cudaError_t launch_direct_verify(const DirectVerify &v, unsigned nmatch, cudaStream_t s);
// C1 = #{x : row_1 . x = d_1} into out[0..1] (low, high 64 bits); buf holds
// 2 (d1 + 1) 128-bit counters.
cudaError_t launch_c1_dp(const int32_t *a1, int n, int d1, void *buf, unsigned long long *out, cudaStream_t s);

}  // namespace msp
