// Shared declarations of the direct pass (direct_join.cu: the class joins,
// direct_kernels.cu: list builds, verification and C1, direct.cu: host
// side).  The direct pass joins residue classes of about 2^13 records per
// side entirely in shared memory; direct_kernels.cu describes the method.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "checked.cuh"

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

// The outer quarter of one side of one instance (at most 9 columns): its
// column tables and where its subset lists go.  Subset u's key is the sum of
// its columns' keys (right side: kd minus it), its class likewise (masked),
// its packed vector the sum of the packed columns, and its mask u.
constexpr int kOuterColsMax = 9;
struct OuterSeg {
  uint32_t ck[kOuterColsMax];     // 32-bit key of each column
  uint32_t cc[kOuterColsMax];     // class contribution of each column
  uint64_t pc[kOuterColsMax][4];  // packed column vectors (16-bit row fields)
  int q;                          // columns
  int neg;                        // 1: key kd - K, class cd - kappa (right side)
  uint32_t kd, cd, cmask;
  uint32_t *okey, *ocls, *omask;  // [2^q]
  uint64_t *ovec;                 // [2^q][4]
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
  uint32_t ni;           // inner subsets (the bound of the MSP_CHECKED checks)
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
// Inner list of one instance by windows of 2^logW classes: the q inner
// columns split into h low and hq high ones; the low subsets, bucketed by
// class at a granularity of 2^gshift classes, and the high subsets'
// keys and classes are built first.
constexpr int kWinBits = 9;            // classes per window (fewer when B < 9)
constexpr int kHighMax = 10;           // high columns
constexpr uint32_t kWinCap = 12288;    // subsets staged per window (mean 2^(q - B) per class)
struct WinBuild {
  int B;
  uint32_t cmask;
  int h, hq;                  // low and high columns
  int logW, gshift;
  uint32_t nc;                // coarse buckets, 2^(B - gshift)
  const uint4 *low;           // [2^h] (key, mask, class, 0) by coarse bucket
  const uint32_t *loff;       // [nc + 1] coarse bucket starts
  const uint32_t *hkey, *hcls;  // [2^hq]
  uint32_t *cnt;              // [2^B] class counts (first pass)
  const uint32_t *ioff;       // [2^B + 1] bucket starts (second pass)
  uint32_t *ikey, *imask;     // [2^q] the list (second pass)
};
// Low subsets (g.q = h) counted by coarse bucket (low == nullptr) or placed
// at the cursors cnt_or_cur.
cudaError_t launch_win_low(const InnerGen &g, int gshift, uint32_t *cnt_or_cur, uint4 *low, cudaStream_t s);
cudaError_t launch_win_high(const InnerGen &g, int h, int hq, uint32_t *hkey, uint32_t *hcls, cudaStream_t s);
// One block per window: class counts (place = false) or placement.
cudaError_t launch_win(const WinBuild &w, bool place, cudaStream_t s);
// Counts by class (scatter = false) or placement at the cursors of the
// inner quarters of every segment of a batch (all of q columns).
cudaError_t launch_direct_inner_batch(const InnerSeg *segs, int nseg, int q, bool scatter, cudaStream_t s);
// Outer lists of nseg segments (device array), one block per segment.
cudaError_t launch_direct_outer(const OuterSeg *segs, int nseg, cudaStream_t s);
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
