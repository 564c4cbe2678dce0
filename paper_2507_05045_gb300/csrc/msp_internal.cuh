// Internal declarations shared by the libmsp translation units.
//
// Vocabulary (Section 2, Algorithm 1): the n columns are cut into quarters
// Q1..Q4 (the paper's A, B, C, D).  Every subset of a quarter is an element
// of that quarter's list, enumerated in Gray-code order t -> g(t) = t^(t>>1).
// The left half-pairs L = Q1 x Q3 and right half-pairs R = Q2 x Q4 are the
// two lists that are joined; x = l u r solves A x = d iff
//     v(l) = d - v(r)                                        (all m rows)
// where v(.) is the vector of the m row sums.
//
// Keys.  Every vector v gets K(v) = sum_i w_i v_i mod 2^64 for fixed odd
// 64-bit weights w_i.  K is additive, so K(a + b) = K(a) + K(b): a left
// record is K(a) + K(b), a right record is K(d) - K(c) - K(e), and matching
// records have equal keys.  Like the paper's hash encoding of the partial
// vectors (Algorithm 4) a key match is only a filter: each one is verified
// exactly on all m packed row sums.
//
// Residue classes.  kappa(v) = (v_1 + sum_{1<i<=t} c_i v_i) mod 2^B is the
// residue of row 1 (t = 1) or of a surrogate combination of rows 1..t (eq. 2
// with odd multipliers c_i instead of powers of nD).  kappa is additive mod
// 2^B, so class r of L is the union over buckets u of Q1[u] x Q3[r - u],
// and class r of R the union of Q2'[u] x Q4'[r - u] with Q2' and Q4' holding
// the transformed values kappa(d) - kappa(c) and -kappa(e).  Only records of
// equal class can match, so classes are independent units of work.
#pragma once

#include "checked.cuh"

#include <cstdint>
#include <cuda_runtime.h>

namespace msp {

constexpr int kMaxRows = 16;      // 16-bit fields, 4 per 64-bit word
constexpr int kMaxVecWords = 4;
constexpr int kMaxN = 100;
constexpr int kMaxStreamClassBits = 27;  // residue classes of the streaming and exact passes
constexpr int kMaskWords = 2;     // n <= 128 fits two words
constexpr int kMaxClassRows = 4;

// Instance constants copied to every kernel by value.
struct InstanceConst {
  int m, n, W;                    // W = ceil(m / 4) packed words
  int q[4], col0[4];              // quarter sizes and first columns
  uint64_t w_row[kMaxRows];       // key weights w_i
  uint32_t c_row[kMaxClassRows];  // class multipliers (c_1 = 1)
  int t_rows;                     // rows in the class key
  int class_bits;                 // B
  uint64_t dvec[kMaxVecWords];    // packed right-hand side
  uint64_t kd;                    // K(d)
  uint32_t cd;                    // kappa(d)
};

// One quarter list in Gray order (index t = Gray rank).
struct QuarterDev {
  int q;
  int64_t size;        // 2^q
  uint64_t *vec;       // [W][size] packed row sums
  uint64_t *key;       // [size]
  uint32_t *cls;       // [size]
  uint32_t *v1;        // [size] row-1 sum
};

// A list sorted by class (counting sort), with its transformed keys.
struct BucketDev {
  int64_t size;
  uint64_t *key;       // [size] transformed key
  uint32_t *cls;       // [size] transformed class
  uint32_t *idx;       // [size] Gray rank in the quarter
  uint32_t *off;       // [M + 1] bucket starts
};

// The generator of one side: outer list (bucketed) x inner list (bucketed).
struct SideGen {
  const uint64_t *okey;
  const uint32_t *ocls;
  int64_t osize;
  const uint64_t *ikey;
  const uint32_t *ioff;
  int64_t isize;        // inner list entries (the bound of the MSP_CHECKED checks)
  int64_t slice_outer;  // outer elements per slice
  int slices;           // slices per class
  int wmax;             // outer elements per window of the streaming scatter
};

struct PassDev {
  SideGen side[2];
  uint32_t cmask;       // 2^B - 1
  int c0;               // first class of the pass
  int nclass;           // classes in the pass
  int D;                // digit bits (top bits of the key)
  int S;                // local sort bits (next bits below the digit)
  // per side: counts / offsets [nclass][slices][2^D]
  uint32_t *cnt[2];
  uint64_t *segstart[2];  // [nclass][2^D] relative to class base
  uint32_t *seglen[2];    // [nclass][2^D]
  uint64_t *classtot[2];  // [nclass]
  uint64_t *classbase[2]; // [nclass] absolute record offset
  uint64_t *rec[2];       // record buffers
  // join outputs
  uint64_t *match_key;    // [match_cap]
  uint32_t *match_cls;    // [match_cap]
  unsigned long long *match_count;
  uint64_t match_cap;
  uint32_t *big_list;     // [big_cap] oversize segments (class_local << 16 | digit)
  unsigned int *big_count;
  uint32_t big_cap;
};

// Streaming pass (fastpath.cu): partitions of fixed capacity <= kFastCap.
constexpr int kFastCap = 4608;

// One instance of a streaming pass (device table; a single solve has one
// entry, a batch one per instance of the same (m, n)).
struct FastInst {
  SideGen side[2];
  const uint64_t *class_base[2];  // [M] first record of each class region (by class id)
  const uint32_t *cap[2];         // [M] records per partition (multiple of 16)
  uint32_t *fill[2];              // [nclass of the pass][2^D] records appended (zeroed per pass)
  uint32_t tag;                   // added to the class id of emitted matches (instance * M)
};

constexpr uint64_t kDefaultWaitNs = 2000000000ull;  // bounded waits of the streaming join: 2 s
struct FastPass {
  const FastInst *inst;           // [ninst] in device memory
  int ninst;
  int slices[2];                  // slices per class and side (same for every instance)
  uint32_t cmask;
  int c0, nclass;                 // classes [c0, c0 + nclass) of every instance
  int D, S;
  uint64_t *rec[2];
  unsigned int *overflow;         // [ninst]: the instance dropped a record (partition full)
  unsigned int *error;            // a bounded wait gave up
  uint64_t wait_ns;               // limit of each bounded wait of the join
  int wait_check;                 // 1: every join block first waits on a phase no copy completes
  uint64_t *match_key;
  uint32_t *match_cls;            // tag + class
  unsigned long long *match_count;
  uint64_t match_cap;
};
// out[i] = exact size of class rbeg + i, i < rcount (classes mod M).
// The same from the classes of the no outer elements (cheaper when no < M).
cudaError_t launch_class_sizes_elems(const uint32_t *ocls, int64_t no, const uint32_t *offI, uint32_t M,
                                     uint32_t rbeg, uint32_t rcount, unsigned long long *out, cudaStream_t s);
cudaError_t launch_class_sizes(const uint32_t *offO, const uint32_t *offI, uint32_t M, uint32_t rbeg,
                               uint32_t rcount, unsigned long long *out, cudaStream_t s);
cudaError_t launch_scatter_fast(const FastPass &p, int nclass_run, cudaStream_t s);
cudaError_t launch_join_fast(const FastPass &p, int nclass_run, cudaStream_t s);
size_t scatter_fast_smem(int D);
// Outer elements per scatter window for an inner list of inner_size
// elements spread over `classes` buckets.
int scatter_window(int64_t inner_size, uint32_t classes);
size_t join_fast_smem();

constexpr int kJoinCap = 6144;   // records per side held in shared memory
constexpr int kJoinThreads = 512;
constexpr int kGenThreads = 256;

// -------------------------------------------------------------------------
// kernels.cu launchers (all asynchronous on `s`; return cudaGetLastError()).
// -------------------------------------------------------------------------
cudaError_t launch_gray(const InstanceConst &ic, const uint64_t *pcol, const uint64_t *kcol,
                        const uint32_t *ccol, const QuarterDev &qd, int col0, cudaStream_t s);
cudaError_t launch_count_classes(const uint32_t *cls, int64_t size, uint32_t mul, uint32_t add,
                                 uint32_t cmask, uint32_t *hist, cudaStream_t s);
cudaError_t launch_bucket_scatter(const QuarterDev &qd, int64_t mul, uint64_t kadd, uint32_t cadd,
                                  uint32_t cmask, uint32_t *cursor, const BucketDev &bd, cudaStream_t s);
cudaError_t launch_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *tmp, cudaStream_t s);
cudaError_t launch_v1_hist(const uint32_t *v1, int64_t size, unsigned long long *hist, cudaStream_t s);
cudaError_t launch_row1_candidates(const unsigned long long *h1, const unsigned long long *h3, int len13,
                                   const unsigned long long *h2, const unsigned long long *h4, int len24,
                                   unsigned long long *hl, unsigned long long *hr, int lenl, int lenr,
                                   int64_t d1, unsigned long long *out2, cudaStream_t s);
cudaError_t launch_gen_count(const PassDev &p, cudaStream_t s);
cudaError_t launch_counts_to_offsets(const PassDev &p, cudaStream_t s);
cudaError_t launch_gen_scatter(const PassDev &p, int nclass_run, cudaStream_t s);
cudaError_t launch_join(const PassDev &p, int nclass_run, cudaStream_t s);
cudaError_t launch_join_big(const PassDev &p, int nclass_run, cudaStream_t s);

// Recovery of the quarter elements behind each matched key, then exact
// verification (Algorithm 2's "if Ax = d").
struct RecoverDev {
  const uint64_t *match_key;
  const uint32_t *match_cls;
  uint64_t nmatch;
  SideGen side[2];
  const uint32_t *oidx[2];  // Gray ranks of the bucketed outer lists
  const uint32_t *iidx[2];  // ... and inner lists
  uint32_t cmask;
  unsigned long long *cand_count[2];  // [nmatch]
  unsigned long long *cand_off[2];    // [nmatch + 1]
  unsigned long long *cand_cur[2];    // [nmatch]
  uint64_t *cand[2];                  // packed (outer gray << 32 | inner gray)
  uint32_t *cand_match[2];            // match id of each candidate (L side)
  uint64_t cand_cap[2];
};
cudaError_t launch_recover(const RecoverDev &r, bool emit, cudaStream_t s);
cudaError_t launch_scan_u64(const unsigned long long *in, unsigned long long *out, int64_t n,
                            unsigned long long *tmp, cudaStream_t s);

struct VerifyDev {
  InstanceConst ic;
  const uint64_t *qvec[4];           // packed vectors of Q1..Q4 (Gray order)
  int64_t qsize[4];
  const uint64_t *candL;
  const uint32_t *candL_match;
  uint64_t nL;
  const uint64_t *candR;
  const unsigned long long *candR_off;  // [nmatch + 1]
  uint64_t *sol;                    // [sol_cap][2]
  unsigned long long *sol_count;
  unsigned long long *pairs_checked;
  uint64_t sol_cap;
};
cudaError_t launch_verify(const VerifyDev &v, cudaStream_t s);

}  // namespace msp
