// Direct pass of libmsp (sm_103a): residue classes small enough that one
// thread block joins a whole class in shared memory, so no half-pair record
// is ever written to device memory.
//
// Split.  The columns are cut into a left half (L, the first ceil(n/2)) and a
// right half (R).  Each half is split again into an OUTER quarter of at most
// 2^10 subsets and an INNER quarter of up to 2^31 subsets: the four lists of
// Algorithm 1 (Section 2) with very uneven sizes, which leaves |L| and |R|,
// and so the work, unchanged.
//
// Classes.  kappa (the residue of row 1, or of a surrogate combination of
// the first rows, eq. 2) is taken mod 2^B with B chosen so that an inner
// residue bucket holds about 16 subsets.  Class r of L is the union over the
// outer subsets a of {a} x Qi[r - kappa(a)]: about 2^13 records, each outer
// subset contributing a run of consecutive keys of the bucketed inner list.
// R uses the transformed lists kappa(d) - kappa(c), -kappa(e) (as in the
// streaming pass), so a pair can only solve A x = d if both halves lie in
// the same class.
//
// Keys.  A record's key is the low 32 bits of the additive key
// K(v) = sum_i w_i v_i of the streaming pass: K(a) + K(b) on the left,
// K(d) - K(c) - K(e) on the right.  Equal vectors give equal keys; a key
// match is only a filter (like the hash encoding of Algorithm 4) and every
// match is verified exactly on all m rows.
//
//   direct_inner_count/scatter_kernel  build the bucketed inner lists
//                       (counting sort of all 2^qi subsets by class; each
//                       thread walks a chunk of subsets in Gray order).
//   direct_join_kernel  persistent blocks take runs of consecutive classes
//                       from a work counter; per class the L keys are
//                       inserted into a shared open-addressing table, then
//                       the R keys probe it; a matched (class, key) is
//                       appended to a device list.
//   direct_verify_kernel one block per matched (class, key): finds every
//                       L pair (a, b) and R pair (c, e) with that key by
//                       scanning the class's inner buckets, and checks each
//                       of their combinations on all m rows (Algorithm 2's
//                       "if A x = d").
//   c1_dp_kernel        C1 = #{x : row_1 . x = d_1}, the number of row-1
//                       candidate pairs the solve rules on (subset-sum
//                       counting over row 1, 128-bit).
#include "host_internal.h"
#include "host_util.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace msp {

namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr int kDT = 512;                  // threads per join block
constexpr int kDW = kDT / 32;             // warps per join block
constexpr int kOuterMax = 32 * kDW;       // outer subsets per side: one per lane of each warp
constexpr int kInnerMax = 31;             // inner quarter columns (32-bit positions)
constexpr int kGenChunk = 6;              // Gray walk of 2^6 subsets per thread

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }


struct InnerGen {
  uint32_t ck[kInnerMax];  // 32-bit key of each column (row sums weighted by w_i)
  uint32_t cc[kInnerMax];  // class contribution of each column (unmasked)
  int q;                   // columns of the quarter
  int neg;                 // 1: store -K and -kappa (right inner list)
  uint32_t cmask;
};

// Subsets of a chunk of 2^c consecutive masks in Gray order: the mask of
// step i is base | g(i), g(i) = i ^ (i >> 1).  f(mask, key, class).
template <typename F>
__device__ __forceinline__ void walk_chunk(const InnerGen &g, uint32_t base, int c, F &&f) {
  uint32_t key = 0, cls = 0;
  for (uint32_t b = base; b; b &= b - 1) {
    const int j = __ffs(b) - 1;
    key += g.ck[j];
    cls += g.cc[j];
  }
  uint32_t gray = 0;
  const uint32_t steps = 1u << c;
  for (uint32_t i = 0; i < steps; ++i) {
    if (i) {
      const int j = __ffs(i) - 1;
      gray ^= 1u << j;
      if (gray & (1u << j)) {
        key += g.ck[j];
        cls += g.cc[j];
      } else {
        key -= g.ck[j];
        cls -= g.cc[j];
      }
    }
    const uint32_t k = g.neg ? 0u - key : key;
    const uint32_t r = (g.neg ? 0u - cls : cls) & g.cmask;
    f(base | gray, k, r);
  }
}

__global__ void direct_inner_count_kernel(InnerGen g, int c, uint64_t nchunks, uint32_t *cnt) {
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < nchunks;
       t += (uint64_t)gridDim.x * blockDim.x) {
    walk_chunk(g, static_cast<uint32_t>(t << c), c, [&](uint32_t, uint32_t, uint32_t r) { atomicAdd(cnt + r, 1u); });
  }
}

__global__ void direct_inner_scatter_kernel(InnerGen g, int c, uint64_t nchunks, uint32_t *cur, uint32_t *ikey,
                                            uint32_t *imask) {
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < nchunks;
       t += (uint64_t)gridDim.x * blockDim.x) {
    walk_chunk(g, static_cast<uint32_t>(t << c), c, [&](uint32_t mask, uint32_t k, uint32_t r) {
      const uint32_t pos = atomicAdd(cur + r, 1u);
      ikey[pos] = k;
      imask[pos] = mask;
    });
  }
}

// The inner quarter of one side of one instance of a batch: its column
// tables and its lists.
struct InnerSeg {
  InnerGen g;
  uint32_t *cnt;    // [2^B] counts, then insertion cursors
  uint32_t *ioff;   // [2^B + 1] bucket starts
  uint32_t *ikey;   // [2^q] keys in bucket order
  uint32_t *imask;  // [2^q] subset masks in bucket order
};

// Counts (scatter = false) or bucket placement (scatter = true) of the inner
// subsets of every segment of a batch: thread t walks chunk t mod
// chunks_per_seg of segment t / chunks_per_seg.
template <bool kScatter>
__global__ void direct_inner_batch_kernel(const InnerSeg *segs, int c, uint64_t chunks_per_seg, uint64_t total) {
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t sg = t / chunks_per_seg;
    const InnerSeg &S = segs[sg];
    const uint32_t base = static_cast<uint32_t>((t - sg * chunks_per_seg) << c);
    if constexpr (kScatter) {
      walk_chunk(S.g, base, c, [&](uint32_t mask, uint32_t k, uint32_t r) {
        const uint32_t pos = atomicAdd(S.cnt + r, 1u);
        S.ikey[pos] = k;
        S.imask[pos] = mask;
      });
    } else {
      walk_chunk(S.g, base, c, [&](uint32_t, uint32_t, uint32_t r) { atomicAdd(S.cnt + r, 1u); });
    }
  }
}

// Bucket starts of every segment of a batch, one block per segment:
// ioff = exclusive scan of the counts (ioff[M] = 2^q), and the counts are
// replaced by the starts (the insertion cursors of the placement pass).
__global__ void __launch_bounds__(1024) direct_inner_offsets_kernel(const InnerSeg *segs, uint32_t M) {
  __shared__ uint32_t wt[32];
  const InnerSeg &S = segs[blockIdx.x];
  const uint32_t per = (M + blockDim.x - 1) / blockDim.x;
  const uint32_t b0 = min(M, threadIdx.x * per), b1 = min(M, b0 + per);
  uint32_t sum = 0;
  for (uint32_t i = b0; i < b1; ++i) sum += S.cnt[i];
  // block exclusive scan of the per-thread sums
  const uint32_t ln = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, x, o);
    if (ln >= static_cast<uint32_t>(o)) x += y;
  }
  if (ln == 31) wt[wp] = x;
  __syncthreads();
  if (wp == 0) {
    uint32_t t = ln < nw ? wt[ln] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, t, o);
      if (ln >= static_cast<uint32_t>(o)) t += y;
    }
    if (ln < nw) wt[ln] = t;
  }
  __syncthreads();
  uint32_t run = x - sum + (wp ? wt[wp - 1] : 0u);
  for (uint32_t i = b0; i < b1; ++i) {
    const uint32_t cnt = S.cnt[i];
    S.ioff[i] = run;
    S.cnt[i] = run;
    run += cnt;
  }
  if (threadIdx.x == blockDim.x - 1) S.ioff[M] = wt[nw - 1];
}

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

constexpr int kQueue = 64;  // deferred keys per warp

// Shared join structures of a block, for a table of 2^TB slots:
//   T     2^TB key slots in buckets of 8 (bucket = top TB - 3 key bits);
//   C     one 16-bit fill counter per bucket, two per word;
//   F     a filter of 2^(TB + 3) bits (bit = top TB + 3 key bits) set for
//         every left key, so that most right keys are settled by one load;
//   claim one bit per slot: the slot's key was already reported.
// T is never cleared: a bucket's slots past its counter are not read.
__host__ __device__ constexpr uint32_t tab_words(int TB) { return 1u << TB; }
__host__ __device__ constexpr uint32_t cnt_words(int TB) { return 1u << (TB - 4); }
__host__ __device__ constexpr uint32_t filt_words(int TB) { return 1u << (TB - 2); }
__host__ __device__ constexpr uint32_t claim_words(int TB) { return 1u << (TB - 5); }

size_t direct_smem_bytes(int TB, int noL, int noR) {
  (void)noL;
  (void)noR;
  return (size_t)4 * (tab_words(TB) + cnt_words(TB) + filt_words(TB) + claim_words(TB))
         + (size_t)kDW * 32 * 8         // per-warp element table
         + (size_t)kDW * 32 * 4         // per-warp start bitmaps
         + (size_t)kDW * kQueue * 4     // per-warp deferred keys
         + (size_t)kDW * 4              // per-warp left totals
         + 16;
}

// Matched (class, key) appended with one atomic per warp.
__device__ __forceinline__ void emit_match(const DirectPass &p, bool e, uint32_t key, uint32_t cls) {
  const uint32_t bal = __ballot_sync(kFull, e);
  if (!bal) return;
  const int leader = __ffs(bal) - 1;
  unsigned long long base = 0;
  if (static_cast<int>(lane_id()) == leader) base = atomicAdd(p.match_count, (unsigned long long)__popc(bal));
  base = __shfl_sync(kFull, base, leader);
  if (e) {
    const unsigned long long slot = base + __popc(bal & ((1u << lane_id()) - 1u));
    if (slot < p.match_cap) {
      p.match_key[slot] = key;
      p.match_cls[slot] = cls;
    }
  }
}

// Every record of one group of 32 outer subsets (lane = subset: bucket
// [st, st + len) of the inner list, outer key ka) whose group-local index
// lies in [lo, hi) is handed to f(okm, key) in batches of kBatch records per
// lane: key[b] is the join key of record i0 + 32 b + lane, bit b of okm says
// whether that record exists.  f is called by all lanes of the warp.  The
// inner keys of the next batch are loaded before f runs on the current one,
// so their latency overlaps the table work.
// Record k belongs to the last nonempty subset whose first record is <= k;
// a bitmap marks the first records (1024 records per segment, one word per
// lane) and a compacted per-warp table holds (start - first record, ka).
constexpr int kBatch = 4;
constexpr bool kPipe = false;  // load the next batch before working on this one

template <typename F>
__device__ __forceinline__ void group_records(uint32_t st, uint32_t len, uint32_t ka,
                                              const uint32_t *__restrict__ ikey, uint2 *et_w, uint32_t *bm_w,
                                              uint32_t lo, uint32_t hi, F &&f) {
  const uint32_t ln = lane_id();
  const uint32_t ltmask = (1u << ln) - 1u;
  const uint32_t lemask = ltmask | (1u << ln);
  uint32_t incl = len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, incl, o);
    if (ln >= static_cast<uint32_t>(o)) incl += y;
  }
  const uint32_t tot = __shfl_sync(kFull, incl, 31);
  const uint32_t pre = incl - len;
  const uint32_t ke = min(hi, tot);
  if (lo >= ke) return;  // warp-uniform
  const uint32_t ne = __ballot_sync(kFull, len != 0);
  __syncwarp();  // earlier readers of et_w are done
  if (len) et_w[__popc(ne & ltmask)] = make_uint2(st - pre, ka);
  for (uint32_t S = lo & ~31u; S < ke; S += 1024u) {
    __syncwarp();
    if (len && pre >= S && pre - S < 1024u) atomicOr(bm_w + ((pre - S) >> 5), 1u << ((pre - S) & 31u));
    __syncwarp();
    const uint32_t myw = bm_w[ln];
    __syncwarp();
    bm_w[ln] = 0u;
    const uint32_t before = __popc(__ballot_sync(kFull, len != 0 && pre < S));
    const uint32_t pc = __popc(myw);
    uint32_t wi = pc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, wi, o);
      if (ln >= static_cast<uint32_t>(o)) wi += y;
    }
    const uint32_t wbase = before + wi - pc;
    const uint32_t send = min(ke, S + 1024u);
    // inner key and outer key of each record of the batch at i0
    auto fetch = [&](uint32_t i0, uint32_t (&raw)[kBatch], uint32_t (&ko)[kBatch], uint32_t &okm) {
      okm = 0u;
      const uint32_t w0 = (i0 - S) >> 5;
#pragma unroll
      for (int b = 0; b < kBatch; ++b) {
        const uint32_t w = (w0 + b) & 31u;
        const uint32_t word = __shfl_sync(kFull, myw, w);
        const uint32_t base = __shfl_sync(kFull, wbase, w);
        const uint32_t k = i0 + 32u * b + ln;
        const bool ok = k >= lo && k < send;
        const uint32_t c = base + __popc(word & lemask) - 1u;
        const uint2 e = et_w[ok ? c : 0u];
        // lanes outside the range read inner element 0: every address
        // formed here lies inside the inner list
        raw[b] = __ldg(ikey + (ok ? e.x + k : 0u));
        ko[b] = e.y;
        okm |= static_cast<uint32_t>(ok) << b;
      }
    };
    uint32_t rc[kBatch], kc[kBatch], okc;
    if constexpr (kPipe) fetch(S, rc, kc, okc);
    for (uint32_t i0 = S; i0 < send; i0 += 32u * kBatch) {
      uint32_t key[kBatch];
      if constexpr (kPipe) {
        uint32_t rn[kBatch], kn[kBatch], okn = 0u;
        const bool more = i0 + 32u * kBatch < send;  // warp-uniform
        if (more) fetch(i0 + 32u * kBatch, rn, kn, okn);
#pragma unroll
        for (int b = 0; b < kBatch; ++b) key[b] = kc[b] + rc[b];
        f(okc, key);
        if (more) {
#pragma unroll
          for (int b = 0; b < kBatch; ++b) {
            rc[b] = rn[b];
            kc[b] = kn[b];
          }
          okc = okn;
        }
      } else {
        fetch(i0, rc, kc, okc);
#pragma unroll
        for (int b = 0; b < kBatch; ++b) key[b] = kc[b] + rc[b];
        f(okc, key);
      }
    }
  }
}

template <int TB>
__global__ void __launch_bounds__(kDT, 2) direct_join_kernel(DirectPass p) {
  constexpr int kBB = TB - 3;        // bucket bits
  constexpr int hshift = 32 - kBB;   // home bucket = top kBB key bits
  constexpr int fshift = 32 - (TB + 3);
  constexpr uint32_t bmask = (1u << kBB) - 1u;
  extern __shared__ __align__(16) uint8_t sm[];
  uint32_t *const T = reinterpret_cast<uint32_t *>(sm);
  uint32_t *const C = T + tab_words(TB);
  uint32_t *const F = C + cnt_words(TB);
  uint32_t *const claim = F + filt_words(TB);
  uint2 *const et = reinterpret_cast<uint2 *>(claim + claim_words(TB));
  uint32_t *const wbm = reinterpret_cast<uint32_t *>(et + kDW * 32);
  uint32_t *const wq = wbm + kDW * 32;      // [kDW][kQueue]
  uint32_t *const wtot = wq + kDW * kQueue;
  const int noL = p.no[0], noR = p.no[1];
  // per-class totals, double-buffered by class parity: class i accumulates
  // into slot i & 1 before its first barrier, and the other slot is reset
  // after that barrier, once every thread has read it for class i - 1
  __shared__ unsigned long long s_fill[2][2];
  __shared__ uint32_t s_bad[2];
  __shared__ uint32_t s_item;
  __shared__ DirectInst s_inst;

  const uint32_t ln = lane_id(), wp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kDW * 32; i += kDT) wbm[i] = 0u;
  // counters, filter and claim bits are contiguous: one pass clears them
  auto clear_table = [&]() {
    constexpr uint32_t n4 = (cnt_words(TB) + filt_words(TB) + claim_words(TB)) / 4;
    uint4 *c4 = reinterpret_cast<uint4 *>(C);
    for (uint32_t i = threadIdx.x; i < n4; i += kDT) c4[i] = make_uint4(0u, 0u, 0u, 0u);
  };
  clear_table();
  if (threadIdx.x < 2) {
    s_fill[threadIdx.x][0] = s_fill[threadIdx.x][1] = 0;
    s_bad[threadIdx.x] = 0;
  }
  uint2 *const et_w = et + wp * 32;
  uint32_t *const bm_w = wbm + wp * 32;
  uint32_t *const q_w = wq + wp * kQueue;
  const uint32_t ltmask = (1u << ln) - 1u;
  uint32_t qn = 0;  // deferred keys of this warp (warp-uniform)
  // Count-claimed slot: the previous fill of bucket b (one 16-bit counter).
  auto take_slot = [&](uint32_t b) -> uint32_t {
    const uint32_t sh = (b & 1u) << 4;
    return (atomicAdd(C + (b >> 1), 1u << sh) >> sh) & 0xffffu;
  };
  auto count_of = [&](uint32_t b) -> uint32_t { return (C[b >> 1] >> ((b & 1u) << 4)) & 0xffffu; };
  // A left key goes to the first slot its counter hands out; a key that
  // finds its bucket full moves on to the next bucket (counting it there
  // too), so a bucket whose counter passed 8 sends probes on as well.
  auto drain_insert = [&]() {
    __syncwarp();
    for (uint32_t i = ln; i < qn; i += 32) {
      const uint32_t key = q_w[i];
      uint32_t b = ((key >> hshift) + 1u) & bmask;  // the home bucket was full
      for (;;) {
        const uint32_t sl = take_slot(b);
        if (sl < 8u) {
          T[8u * b + sl] = key;
          break;
        }
        b = (b + 1u) & bmask;
      }
    }
    __syncwarp();
    qn = 0;
  };
  auto claim_slot = [&](uint32_t slot) -> bool {
    const uint32_t bit = 1u << (slot & 31u);
    return (atomicOr(claim + (slot >> 5), bit) & bit) == 0u;
  };
  // A right key that passed the filter: the first slot holding it, walking
  // from its home bucket while buckets have sent keys on.
  auto drain_probe = [&](uint32_t r) {
    __syncwarp();
    for (uint32_t i0 = 0; i0 < qn; i0 += 32) {
      const uint32_t i = i0 + ln;
      bool first = false;
      uint32_t key = 0;
      if (i < qn) {
        key = q_w[i];
        uint32_t b = key >> hshift;
        for (;;) {
          const uint32_t c = count_of(b);
          const uint4 *s4 = reinterpret_cast<const uint4 *>(T + 8u * b);
          const uint4 u = s4[0], v = s4[1];
          const uint32_t x[8] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w};
          uint32_t hit = 8u;
#pragma unroll
          for (int j = 7; j >= 0; --j)
            if (static_cast<uint32_t>(j) < c && x[j] == key) hit = j;
          if (hit < 8u) {
            first = claim_slot(8u * b + hit);
            break;
          }
          if (c <= 8u) break;
          b = (b + 1u) & bmask;
        }
      }
      emit_match(p, first, key, r);
    }
    __syncwarp();
    qn = 0;
  };
  // warp-collective: append the lanes' deferred keys
  auto defer = [&](bool want, uint32_t key) -> bool {
    const uint32_t bal = __ballot_sync(kFull, want);
    if (!bal) return false;
    if (want) q_w[qn + __popc(bal & ltmask)] = key;
    qn += __popc(bal);
    return qn >= 32u;
  };
  const uint32_t cmask = p.cmask;
  const uint32_t *__restrict__ ioffL = nullptr;
  const uint32_t *__restrict__ ioffR = nullptr;
  const uint32_t *__restrict__ ikeyL = nullptr;
  const uint32_t *__restrict__ ikeyR = nullptr;
  const uint32_t per_inst = (p.nclass + p.chunk - 1) / p.chunk;  // work items per instance
  const uint32_t nitems = per_inst * p.ninst;
  unsigned long long my_records = 0;  // thread 0 only
  // this lane's outer subset (key, class) on both sides, for the current
  // instance; bucket bounds [ioff[w], ioff[w + 1]) of it for a class (0, 0
  // past the outer list)
  const int el = wp * 32 + ln;
  uint32_t kaL = 0, kaR = 0, clL = 0, clR = 0;
  uint32_t cur_inst = 0xffffffffu;
  uint32_t pfL0 = 0, pfL1 = 0, pfR0 = 0, pfR1 = 0;
  auto load_bounds = [&](uint32_t r) {
    pfL0 = pfL1 = pfR0 = pfR1 = 0u;
    if (el < noL) {
      const uint32_t w = (r - clL) & cmask;
      pfL0 = ioffL[w];
      pfL1 = ioffL[w + 1];
    }
    if (el < noR) {
      const uint32_t w = (r - clR) & cmask;
      pfR0 = ioffR[w];
      pfR1 = ioffR[w + 1];
    }
  };
  uint32_t par = 0;                   // parity of the block's class count

  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t it = atomicAdd(p.work, 1u);
      s_item = it;
      if (it < nitems) s_inst = p.inst[it / per_inst];
    }
    __syncthreads();
    const uint32_t item = s_item;
    if (item >= nitems) break;
    const uint32_t ii = item / per_inst;
    if (ii != cur_inst) {  // block-uniform
      cur_inst = ii;
      ioffL = s_inst.side[0].ioff;
      ioffR = s_inst.side[1].ioff;
      ikeyL = s_inst.side[0].ikey;
      ikeyR = s_inst.side[1].ikey;
      kaL = el < noL ? s_inst.side[0].okey[el] : 0u;
      clL = el < noL ? s_inst.side[0].ocls[el] : 0u;
      kaR = el < noR ? s_inst.side[1].okey[el] : 0u;
      clR = el < noR ? s_inst.side[1].ocls[el] : 0u;
    }
    const uint32_t tag = ii << p.class_bits;
    const uint32_t rb = (item - ii * per_inst) * p.chunk, re = min(p.nclass, rb + p.chunk);
    for (uint32_t ri = rb; ri < re; ++ri, par ^= 1u) {
      const uint32_t r = (p.c0 + ri) & cmask;
      // ---- bucket of this warp's outer subsets (lane = subset), loaded
      //      during the previous class ----
      load_bounds(r);
      const uint32_t stL = pfL0, lnL = pfL1 - pfL0, stR = pfR0, lnR = pfR1 - pfR0;
      unsigned long long sumL = lnL, sumR = lnR;
      bool big = lnL >= (1u << 24) || lnR >= (1u << 24);
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        sumL += __shfl_xor_sync(kFull, sumL, o);
        sumR += __shfl_xor_sync(kFull, sumR, o);
      }
      big = __any_sync(kFull, big);
      if (ln == 0) {
        atomicAdd(&s_fill[par][0], sumL);
        atomicAdd(&s_fill[par][1], sumR);
        wtot[wp] = static_cast<uint32_t>(min(sumL, 0xffffffffull));
        if (big) {
          atomicOr(&s_bad[par], 1u);
          atomicOr(p.error, 1u);
        }
      }
      __syncthreads();
      const unsigned long long TL = s_fill[par][0];
      const unsigned long long TR = s_fill[par][1];
      // a class past 2^31 records on a side, or a bucket past 2^24, is beyond
      // this kernel: it is skipped and the host, seeing the error flag, solves
      // the instance on another path
      const bool skip = s_bad[par] != 0u || TL >= (1ull << 31) || TR >= (1ull << 31);
      if (skip && threadIdx.x == 0) atomicOr(p.error, 1u);
      if (threadIdx.x == 0) {
        my_records += TL + TR;
        s_fill[par ^ 1u][0] = s_fill[par ^ 1u][1] = 0;
        s_bad[par ^ 1u] = 0;
      }
      const uint32_t cap = p.insert_cap;
      const uint32_t nch = skip ? 0u : (TL > cap ? static_cast<uint32_t>((TL + cap - 1) / cap) : 1u);
      uint32_t woff = 0;
      if (nch > 1)
        for (uint32_t w = 0; w < wp; ++w) woff += wtot[w];
      for (uint32_t ch = 0; ch < nch; ++ch) {
        if (ch) {
          __syncthreads();
          clear_table();
          __syncthreads();
        }
        // ---- left records of this table fill: insert ----
        if (wp * 32 < static_cast<uint32_t>(noL)) {  // warp-uniform
          uint32_t lo = 0, hi = 0xffffffffu;
          if (nch > 1) {
            const uint32_t a = ch * cap, b = a + cap;  // global range of this fill
            lo = a > woff ? a - woff : 0u;
            hi = b > woff ? b - woff : 0u;
          }
          group_records(stL, lnL, kaL, ikeyL, et_w, bm_w, lo, hi,
                        [&](uint32_t okm, const uint32_t(&key)[kBatch]) {
#pragma unroll
            for (int b = 0; b < kBatch; ++b) {
              const uint32_t k = key[b];
              const bool ok = (okm >> b) & 1u;
              bool full = false;
              if (ok) {
                const uint32_t fb = k >> fshift;
                atomicOr(F + (fb >> 5), 1u << (fb & 31u));
                const uint32_t hb = k >> hshift;
                const uint32_t sl = take_slot(hb);
                if (sl < 8u)
                  T[8u * hb + sl] = k;
                else
                  full = true;
              }
              if (defer(full, k)) drain_insert();
            }
          });
          if (qn) drain_insert();
        }
        __syncthreads();
        // ---- right records: probe ----
        if (wp * 32 < static_cast<uint32_t>(noR)) {
          group_records(stR, lnR, kaR, ikeyR, et_w, bm_w, 0u, 0xffffffffu,
                        [&](uint32_t okm, const uint32_t(&key)[kBatch]) {
            uint32_t fw[kBatch];
#pragma unroll
            for (int b = 0; b < kBatch; ++b) fw[b] = F[key[b] >> (fshift + 5)];
#pragma unroll
            for (int b = 0; b < kBatch; ++b) {
              const uint32_t k = key[b];
              const bool pass = ((okm >> b) & 1u) && ((fw[b] >> ((k >> fshift) & 31u)) & 1u);
              if (defer(pass, k)) drain_probe(tag | r);
            }
          });
          if (qn) drain_probe(tag | r);
        }
      }
      __syncthreads();
      clear_table();
    }
  }
  if (threadIdx.x == 0 && my_records) atomicAdd(p.records, my_records);
}

// -------------------------------------------------------------------------
// Recovery and exact verification of the matched (class, key) pairs.
// -------------------------------------------------------------------------
constexpr int kVT = 512;  // one thread per outer subset of each side
constexpr int kVCand = 512;

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
  unsigned long long *pairs;
  unsigned int *overflow;    // a match had more candidates than the block holds
};

__device__ __forceinline__ void put_bits(uint64_t &lo, uint64_t &hi, uint64_t bits, int pos) {
  if (pos >= 64) {
    hi |= bits << (pos - 64);
  } else {
    lo |= bits << pos;
    if (pos > 0) hi |= bits >> (64 - pos);
  }
}

__global__ void __launch_bounds__(kVT) direct_verify_kernel(DirectVerify v) {
  static_assert(kVT >= kOuterMax, "one pass over the outer subsets");
  __shared__ uint2 cand[2][kVCand];
  __shared__ uint32_t ncand[2];
  __shared__ uint64_t scol[2][kInnerMax][4];
  const uint32_t key = v.match_key[blockIdx.x];
  const uint32_t tagged = v.match_cls[blockIdx.x];
  const uint32_t ii = tagged >> v.class_bits;
  const uint32_t r = tagged & v.cmask;
  const DirectVerifyInst &vi = v.inst[ii];
  if (threadIdx.x < 2) ncand[threadIdx.x] = 0;
  for (int i = threadIdx.x; i < 2 * kInnerMax * 4; i += kVT) {
    const int s = i / (kInnerMax * 4), j = (i / 4) % kInnerMax, w = i % 4;
    scol[s][j][w] = j < v.qi[s] ? vi.icol[s][j * 4 + w] : 0ull;
  }
  __syncthreads();
  // thread a scans the bucket of outer subset a on both sides; the bucket
  // bounds of the two sides are loaded together
  {
    const int a = threadIdx.x;
    uint32_t b0[2] = {0u, 0u}, b1[2] = {0u, 0u}, ka[2] = {0u, 0u};
#pragma unroll
    for (int s = 0; s < 2; ++s)
      if (a < vi.side[s].no) {
        const uint32_t w = (r - vi.side[s].ocls[a]) & v.cmask;
        b0[s] = vi.side[s].ioff[w];
        b1[s] = vi.side[s].ioff[w + 1];
        ka[s] = vi.side[s].okey[a];
      }
#pragma unroll
    for (int s = 0; s < 2; ++s)
      for (uint32_t j = b0[s]; j < b1[s]; ++j)
        if (ka[s] + vi.side[s].ikey[j] == key) {
          const uint32_t slot = atomicAdd(&ncand[s], 1u);
          if (slot < kVCand) cand[s][slot] = make_uint2(static_cast<uint32_t>(a), j);
        }
  }
  __syncthreads();
  const uint32_t nL = min(ncand[0], static_cast<uint32_t>(kVCand));
  const uint32_t nR = min(ncand[1], static_cast<uint32_t>(kVCand));
  if (threadIdx.x == 0) {
    if (ncand[0] > kVCand || ncand[1] > kVCand) atomicOr(v.overflow, 1u);
    atomicAdd(v.pairs, (unsigned long long)nL * nR);
  }
  const uint32_t np = nL * nR;
  for (uint32_t pi = threadIdx.x; pi < np; pi += kVT) {
    const uint2 l = cand[0][pi / nR], rr = cand[1][pi % nR];
    uint64_t vec[4];
    for (int w = 0; w < 4; ++w) vec[w] = vi.ovec[0][l.x * 4 + w] + vi.ovec[1][rr.x * 4 + w];
    const uint32_t mL = vi.imask[0][l.y], mR = vi.imask[1][rr.y];
    for (uint32_t b = mL; b; b &= b - 1) {
      const int j = __ffs(b) - 1;
      for (int w = 0; w < 4; ++w) vec[w] += scol[0][j][w];
    }
    for (uint32_t b = mR; b; b &= b - 1) {
      const int j = __ffs(b) - 1;
      for (int w = 0; w < 4; ++w) vec[w] += scol[1][j][w];
    }
    bool eq = true;
    for (int w = 0; w < v.W; ++w) eq &= vec[w] == vi.dvec[w];
    if (eq) {
      uint64_t lo = 0, hi = 0;
      put_bits(lo, hi, vi.omask[0][l.x], v.col_o[0]);
      put_bits(lo, hi, mL, v.col_i[0]);
      put_bits(lo, hi, vi.omask[1][rr.x], v.col_o[1]);
      put_bits(lo, hi, mR, v.col_i[1]);
      const unsigned long long slot = atomicAdd(v.sol_count, 1ull);
      if (slot < v.sol_cap) {
        v.sol[3 * slot] = lo;
        v.sol[3 * slot + 1] = hi;
        v.sol[3 * slot + 2] = ii;
      }
    }
  }
}

// C1 = number of x in {0,1}^n with row_1 . x = d_1 (128-bit): one block,
// counts over sums 0..d_1 in two device buffers, one column per step.
__global__ void __launch_bounds__(1024) c1_dp_kernel(const int32_t *a1, int n, int d1, unsigned __int128 *buf,
                                                     unsigned long long *out) {
  unsigned __int128 *cur = buf, *nxt = buf + (d1 + 1);
  for (int s = threadIdx.x; s <= d1; s += blockDim.x) cur[s] = s == 0 ? 1 : 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const int a = a1[j];
    for (int s = threadIdx.x; s <= d1; s += blockDim.x) nxt[s] = cur[s] + (s >= a ? cur[s - a] : 0);
    __syncthreads();
    unsigned __int128 *t = cur;
    cur = nxt;
    nxt = t;
  }
  if (threadIdx.x == 0) {
    out[0] = static_cast<unsigned long long>(cur[d1]);
    out[1] = static_cast<unsigned long long>(cur[d1] >> 64);
  }
}

template <int TB>
cudaError_t launch_direct_join_tb(const DirectPass &p, cudaStream_t s) {
  static size_t attr = 0;
  static int per_sm = 0, sms = 0;
  const size_t smem = direct_smem_bytes(TB, p.no[0], p.no[1]);
  if (smem > attr) {
    cudaError_t e = cudaFuncSetAttribute(direct_join_kernel<TB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    attr = smem;
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, direct_join_kernel<TB>, kDT, smem) != cudaSuccess ||
        n < 1) {
      cudaGetLastError();
      n = 1;
    }
    per_sm = n;
  }
  // work items of up to 4 consecutive classes (neighbouring classes share
  // bucket-offset and inner-key sectors; short items keep the blocks
  // evenly loaded to the end of the launch)
  const uint32_t resident = static_cast<uint32_t>(std::max(1, per_sm * sms));
  DirectPass q = p;
  q.chunk = static_cast<uint32_t>(
      std::max<uint64_t>(1, std::min<uint64_t>(4, (uint64_t)p.nclass * p.ninst / (4 * resident))));
  const uint64_t nitems = (uint64_t)((q.nclass + q.chunk - 1) / q.chunk) * q.ninst;
  const int blocks = static_cast<int>(std::max<uint64_t>(1, std::min<uint64_t>(nitems, resident)));
  direct_join_kernel<TB><<<blocks, kDT, smem, s>>>(q);
  return cudaGetLastError();
}

cudaError_t launch_direct_join(int TB, const DirectPass &p, cudaStream_t s) {
  switch (TB) {
    case 12: return launch_direct_join_tb<12>(p, s);
    case 13: return launch_direct_join_tb<13>(p, s);
    case 14: return launch_direct_join_tb<14>(p, s);
    case 15: return launch_direct_join_tb<15>(p, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

// -------------------------------------------------------------------------
// Host side.
// -------------------------------------------------------------------------
DirectPlan make_direct_plan(int m, int n, int table_bits) {
  DirectPlan d{};
  d.m = m;
  d.n = n;
  d.W = (m + 3) / 4;
  d.cols[0] = (n + 1) / 2;
  d.cols[1] = n - d.cols[0];
  const int lg = std::max(d.cols[0], d.cols[1]);
  // about 2^13 records per class and side; inner buckets of about 16
  d.B = std::max(0, lg - 13);
  d.TB = table_bits >= 12 && table_bits <= 15 ? table_bits : 14;
  for (int s = 0; s < 2; ++s) {
    const int c = d.cols[s];
    int qi = std::min(c, d.B + 4);
    int qo = c - qi;
    if (qo > 9) {  // small halves: everything beyond 9 outer columns goes inner
      qo = 9;
      qi = c - qo;
    }
    d.qo[s] = qo;
    d.qi[s] = qi;
  }
  d.col_o[0] = 0;
  d.col_i[0] = d.qo[0];
  d.col_o[1] = d.cols[0];
  d.col_i[1] = d.cols[0] + d.qo[1];
  d.t = std::min(m, d.B <= 6 ? 1 : (d.B <= 14 ? 2 : (d.B <= 21 ? 3 : 4)));
  d.ok = n >= 2 && d.qi[0] <= kInnerMax && d.qi[1] <= kInnerMax && (1 << d.qo[0]) <= kOuterMax &&
         (1 << d.qo[1]) <= kOuterMax && d.B <= 27;
  return d;
}

size_t direct_footprint(const DirectPlan &d) {
  double b = 0;
  for (int s = 0; s < 2; ++s) b += 8.0 * std::ldexp(1.0, d.qi[s]);  // inner keys and masks
  b += 2.0 * 4.0 * (std::ldexp(1.0, d.B) + 1);                       // bucket offsets
  b += 4.0 * (std::ldexp(1.0, d.B) + 1);                             // counts / cursors while building
  b += 12.0 * kDirectMatchCap + (64 << 20);                          // matches, small tables, margin
  return static_cast<size_t>(b);
}

namespace {

// Host and device lists of one instance of a direct pass.
struct DirectLists {
  std::vector<uint32_t> okey[2], ocls[2], omask[2];
  std::vector<uint64_t> ovec[2];
  uint64_t dvec[4] = {0, 0, 0, 0};
  uint32_t *ikey[2] = {nullptr, nullptr}, *imask[2] = {nullptr, nullptr}, *ioff[2] = {nullptr, nullptr};
  uint64_t *icol[2] = {nullptr, nullptr};
  uint32_t *d_okey[2] = {nullptr, nullptr}, *d_ocls[2] = {nullptr, nullptr}, *d_omask[2] = {nullptr, nullptr};
  uint64_t *d_ovec[2] = {nullptr, nullptr};
};

struct Copier {
  msp_stats *st;
  cudaStream_t s;
  cudaError_t h2d(void *dst, const void *src, size_t b) {
    if (st) st->h2d_bytes += b;
    return cudaMemcpyAsync(dst, src, b, cudaMemcpyHostToDevice, s);
  }
  cudaError_t d2h(void *dst, const void *src, size_t b) {
    if (st) st->d2h_bytes += b;
    return cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToHost, s);
  }
};

// S0 + S1 + S2 of one instance: column keys and classes, the outer lists
// (host, at most 2^9 subsets each), the inner lists bucketed by class
// (device: count, offsets, scatter).  `cnt` and `scantmp` are scratch of
// 2^B + 1 and (2^B + 1) / 4096 + 1 entries, shared by successive calls.
// S0 + S1 on the host for one instance: the column keys and classes, the
// outer lists (at most 2^9 subsets each), the packed right-hand side, and
// the column tables g[side] and packed column vectors icol[side] of the
// inner quarters.
void prep_direct_host(const int32_t *A, const int32_t *d, int m, int n, const DirectPlan &dp, const Plan &kp,
                      DirectLists &L, InnerGen g[2], std::vector<uint64_t> icol[2]) {
  const uint32_t M = 1u << dp.B, cmask = M - 1u;
  std::vector<uint32_t> ck(n), cc(n);
  std::vector<uint64_t> pc((size_t)n * 4, 0);
  for (int j = 0; j < n; ++j) {
    uint32_t k = 0, c = 0;
    for (int i = 0; i < m; ++i) {
      const uint32_t a = static_cast<uint32_t>(A[(size_t)i * n + j]);
      k += static_cast<uint32_t>(kp.w_row[i]) * a;
      if (i < dp.t) c += kp.c_row[i] * a;
      pc[(size_t)j * 4 + i / 4] += static_cast<uint64_t>(a) << (16 * (i % 4));
    }
    ck[j] = k;
    cc[j] = c;
  }
  uint32_t kd = 0, cd = 0;
  for (int i = 0; i < m; ++i) {
    const uint32_t di = static_cast<uint32_t>(d[i]);
    kd += static_cast<uint32_t>(kp.w_row[i]) * di;
    if (i < dp.t) cd += kp.c_row[i] * di;
    L.dvec[i / 4] += static_cast<uint64_t>(di) << (16 * (i % 4));
  }
  for (int sd = 0; sd < 2; ++sd) {
    const int q = dp.qo[sd], c0 = dp.col_o[sd];
    const uint32_t no = 1u << q;
    L.okey[sd].resize(no);
    L.ocls[sd].resize(no);
    L.omask[sd].resize(no);
    L.ovec[sd].assign((size_t)no * 4, 0);
    for (uint32_t u = 0; u < no; ++u) {
      uint32_t k = 0, c = 0;
      for (int j = 0; j < q; ++j)
        if (u >> j & 1u) {
          k += ck[c0 + j];
          c += cc[c0 + j];
          for (int w = 0; w < 4; ++w) L.ovec[sd][(size_t)u * 4 + w] += pc[(size_t)(c0 + j) * 4 + w];
        }
      L.okey[sd][u] = sd ? kd - k : k;
      L.ocls[sd][u] = (sd ? cd - c : c) & cmask;
      L.omask[sd][u] = u;
    }
  }
  for (int sd = 0; sd < 2; ++sd) {
    const int q = dp.qi[sd], c0 = dp.col_i[sd];
    g[sd] = InnerGen{};
    for (int j = 0; j < q; ++j) {
      g[sd].ck[j] = ck[c0 + j];
      g[sd].cc[j] = cc[c0 + j];
    }
    g[sd].q = q;
    g[sd].neg = sd;
    g[sd].cmask = cmask;
    icol[sd].assign(pc.begin() + (size_t)c0 * 4, pc.begin() + (size_t)(c0 + q) * 4);
    icol[sd].resize((size_t)std::max(q, 1) * 4, 0);
  }
}

// S0 + S1 + S2 of one instance: host preparation, then the inner lists
// bucketed by class on the device (count, offsets, scatter).  `cnt` and
// `scantmp` are scratch of 2^B + 1 and (2^B + 1) / 4096 + 1 entries, shared
// by successive calls.
int build_direct_lists(const int32_t *A, const int32_t *d, int m, int n, const DirectPlan &dp, const Plan &kp,
                       DevAlloc &da, Copier &cp, Prof &prof, uint32_t *cnt, uint32_t *scantmp, DirectLists &L) {
  cudaStream_t s = cp.s;
  const uint32_t M = 1u << dp.B;
  InnerGen gs[2];
  std::vector<uint64_t> icol[2];
  prep_direct_host(A, d, m, n, dp, kp, L, gs, icol);
  for (int sd = 0; sd < 2; ++sd) {
    const int q = dp.qi[sd];
    const uint64_t ni = uint64_t(1) << q;
    CK(da.get(&L.ikey[sd], ni));
    CK(da.get(&L.imask[sd], ni));
    CK(da.get(&L.ioff[sd], (size_t)M + 1));
    CK(da.get(&L.icol[sd], icol[sd].size()));
    CK(cp.h2d(L.icol[sd], icol[sd].data(), sizeof(uint64_t) * icol[sd].size()));
    const InnerGen &g = gs[sd];
    const int c = std::min(q, kGenChunk);
    const uint64_t nchunks = ni >> c;
    const unsigned blocks = static_cast<unsigned>(std::min<uint64_t>((nchunks + 255) / 256, 1u << 20));
    CK(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * M, s));
    LAUNCH(MSP_K_BUCKET, 1, 0, (direct_inner_count_kernel<<<blocks, 256, 0, s>>>(g, c, nchunks, cnt), cudaGetLastError()));
    LAUNCH(MSP_K_BUCKET, 3, 0, launch_scan_u32(cnt, L.ioff[sd], M, scantmp, s));
    CK(cudaMemcpyAsync(cnt, L.ioff[sd], sizeof(uint32_t) * M, cudaMemcpyDeviceToDevice, s));
    LAUNCH(MSP_K_BUCKET, 1, 0,
           (direct_inner_scatter_kernel<<<blocks, 256, 0, s>>>(g, c, nchunks, cnt, L.ikey[sd], L.imask[sd]),
            cudaGetLastError()));
  }
  for (int sd = 0; sd < 2; ++sd) {
    const size_t no = L.okey[sd].size();
    CK(da.get(&L.d_okey[sd], no));
    CK(da.get(&L.d_ocls[sd], no));
    CK(da.get(&L.d_omask[sd], no));
    CK(da.get(&L.d_ovec[sd], no * 4));
    CK(cp.h2d(L.d_okey[sd], L.okey[sd].data(), 4 * no));
    CK(cp.h2d(L.d_ocls[sd], L.ocls[sd].data(), 4 * no));
    CK(cp.h2d(L.d_omask[sd], L.omask[sd].data(), 4 * no));
    CK(cp.h2d(L.d_ovec[sd], L.ovec[sd].data(), 8 * 4 * no));
  }
  return MSP_OK;
}

// The lists of the instances idx[k] of a batch (all of one (m, n)), built
// together: the host part per instance, then one upload per array kind and,
// per side, one count launch, one offsets launch (one block per instance)
// and one placement launch over the inner quarters of all instances.
int build_direct_lists_batch(const int32_t *const *A, const int32_t *const *d, const std::vector<int> &idx, int m,
                             int n, const DirectPlan &dp, const Plan &kp, DevAlloc &da, Copier &cp, Prof &prof,
                             std::vector<DirectLists> &lists) {
  cudaStream_t s = cp.s;
  const size_t K = idx.size();
  const uint32_t M = 1u << dp.B;
  lists.assign(K, DirectLists{});
  std::vector<InnerSeg> segs(2 * K);  // segment side * K + k
  std::vector<uint64_t> icol_h[2];
  std::vector<uint32_t> ok_h[2], oc_h[2], om_h[2];
  std::vector<uint64_t> ov_h[2];
  for (size_t k = 0; k < K; ++k) {
    InnerGen g[2];
    std::vector<uint64_t> icol[2];
    prep_direct_host(A[idx[k]], d[idx[k]], m, n, dp, kp, lists[k], g, icol);
    for (int sd = 0; sd < 2; ++sd) {
      segs[sd * K + k].g = g[sd];
      icol_h[sd].insert(icol_h[sd].end(), icol[sd].begin(), icol[sd].end());
      ok_h[sd].insert(ok_h[sd].end(), lists[k].okey[sd].begin(), lists[k].okey[sd].end());
      oc_h[sd].insert(oc_h[sd].end(), lists[k].ocls[sd].begin(), lists[k].ocls[sd].end());
      om_h[sd].insert(om_h[sd].end(), lists[k].omask[sd].begin(), lists[k].omask[sd].end());
      ov_h[sd].insert(ov_h[sd].end(), lists[k].ovec[sd].begin(), lists[k].ovec[sd].end());
    }
  }
  for (int sd = 0; sd < 2; ++sd) {
    const uint64_t ni = uint64_t(1) << dp.qi[sd];
    const size_t no = size_t(1) << dp.qo[sd];
    const size_t nic = icol_h[sd].size() / K;
    uint32_t *ikey, *imask, *ioff, *cnt, *okey, *ocls, *omask;
    uint64_t *icol, *ovec;
    CK(da.get(&ikey, ni * K));
    CK(da.get(&imask, ni * K));
    CK(da.get(&ioff, ((size_t)M + 1) * K));
    CK(da.get(&cnt, (size_t)M * K));
    CK(da.get(&icol, icol_h[sd].size()));
    CK(da.get(&okey, no * K));
    CK(da.get(&ocls, no * K));
    CK(da.get(&omask, no * K));
    CK(da.get(&ovec, 4 * no * K));
    CK(cp.h2d(icol, icol_h[sd].data(), 8 * icol_h[sd].size()));
    CK(cp.h2d(okey, ok_h[sd].data(), 4 * no * K));
    CK(cp.h2d(ocls, oc_h[sd].data(), 4 * no * K));
    CK(cp.h2d(omask, om_h[sd].data(), 4 * no * K));
    CK(cp.h2d(ovec, ov_h[sd].data(), 32 * no * K));
    CK(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * M * K, s));
    for (size_t k = 0; k < K; ++k) {
      DirectLists &L = lists[k];
      L.ikey[sd] = ikey + ni * k;
      L.imask[sd] = imask + ni * k;
      L.ioff[sd] = ioff + ((size_t)M + 1) * k;
      L.icol[sd] = icol + nic * k;
      L.d_okey[sd] = okey + no * k;
      L.d_ocls[sd] = ocls + no * k;
      L.d_omask[sd] = omask + no * k;
      L.d_ovec[sd] = ovec + 4 * no * k;
      InnerSeg &S = segs[sd * K + k];
      S.cnt = cnt + (size_t)M * k;
      S.ioff = L.ioff[sd];
      S.ikey = L.ikey[sd];
      S.imask = L.imask[sd];
    }
  }
  InnerSeg *d_segs;
  CK(da.get(&d_segs, 2 * K));
  CK(cp.h2d(d_segs, segs.data(), sizeof(InnerSeg) * 2 * K));
  for (int pass = 0; pass < 2; ++pass) {  // 0: counts, 1: placement
    if (pass == 1) {
      if (M <= (1u << 20)) {
        LAUNCH(MSP_K_BUCKET, 1, 0,
               (direct_inner_offsets_kernel<<<static_cast<unsigned>(2 * K), 1024, 0, s>>>(d_segs, M),
                cudaGetLastError()));
      } else {
        uint32_t *scantmp;
        CK(da.get(&scantmp, ((size_t)M + 1 + 4095) / 4096 + 1));
        for (size_t i = 0; i < 2 * K; ++i) {
          LAUNCH(MSP_K_BUCKET, 3, 0, launch_scan_u32(segs[i].cnt, segs[i].ioff, M, scantmp, s));
          CK(cudaMemcpyAsync(segs[i].cnt, segs[i].ioff, sizeof(uint32_t) * M, cudaMemcpyDeviceToDevice, s));
        }
      }
    }
    for (int sd = 0; sd < 2; ++sd) {
      const int q = dp.qi[sd];
      const int c = std::min(q, kGenChunk);
      const uint64_t per = (uint64_t(1) << q) >> c;
      const uint64_t total = per * K;
      const unsigned blocks = static_cast<unsigned>(std::min<uint64_t>((total + 255) / 256, 1u << 20));
      const InnerSeg *sp = d_segs + sd * K;
      if (pass == 0)
        LAUNCH(MSP_K_BUCKET, 1, 0,
               (direct_inner_batch_kernel<false><<<blocks, 256, 0, s>>>(sp, c, per, total), cudaGetLastError()));
      else
        LAUNCH(MSP_K_BUCKET, 1, 0,
               (direct_inner_batch_kernel<true><<<blocks, 256, 0, s>>>(sp, c, per, total), cudaGetLastError()));
    }
  }
  return MSP_OK;
}

// The class joins and the verification of the instances `lists` (all of one
// (m, n)), over the residue classes [c_begin, c_end) of each.  Solutions go
// to out[instance] as two words each (unsorted); st (may be null) receives
// passes, records, matches and pairs verified.  Returns MSP_OK,
// kDirectFallback, or an error status.
int run_direct(const std::vector<DirectLists> &lists, const DirectPlan &dp, uint32_t c_begin, uint32_t c_end,
               DevAlloc &da, Copier &cp, Prof &prof, msp_stats *st, const volatile int *cancel,
               std::vector<std::vector<uint64_t>> &out) {
  cudaStream_t s = cp.s;
  const uint32_t M = 1u << dp.B, cmask = M - 1u;
  const uint32_t K = static_cast<uint32_t>(lists.size());
  out.assign(K, {});
  if (K == 0 || c_begin >= c_end) return MSP_OK;
  std::vector<DirectInst> tab(K);
  std::vector<DirectVerifyInst> vtab(K);
  for (uint32_t k = 0; k < K; ++k) {
    const DirectLists &L = lists[k];
    for (int sd = 0; sd < 2; ++sd) {
      DirectSide &ds = tab[k].side[sd];
      ds.okey = L.d_okey[sd];
      ds.ocls = L.d_ocls[sd];
      ds.ikey = L.ikey[sd];
      ds.ioff = L.ioff[sd];
      ds.no = static_cast<int>(L.okey[sd].size());
      DirectVerifyInst &vi = vtab[k];
      vi.side[sd] = ds;
      vi.imask[sd] = L.imask[sd];
      vi.omask[sd] = L.d_omask[sd];
      vi.ovec[sd] = L.d_ovec[sd];
      vi.icol[sd] = L.icol[sd];
    }
    for (int w = 0; w < 4; ++w) vtab[k].dvec[w] = L.dvec[w];
  }
  DirectInst *d_tab;
  DirectVerifyInst *d_vtab;
  CK(da.get(&d_tab, K));
  CK(da.get(&d_vtab, K));
  CK(cp.h2d(d_tab, tab.data(), sizeof(DirectInst) * K));
  CK(cp.h2d(d_vtab, vtab.data(), sizeof(DirectVerifyInst) * K));

  uint32_t *match_key, *match_cls;
  unsigned long long *match_count, *records;
  unsigned int *work, *err;
  CK(da.get(&match_key, kDirectMatchCap));
  CK(da.get(&match_cls, kDirectMatchCap));
  CK(da.get(&match_count, 1));
  CK(da.get(&records, 1));
  CK(da.get(&err, 1));
  CK(cudaMemsetAsync(match_count, 0, sizeof(unsigned long long), s));
  CK(cudaMemsetAsync(records, 0, sizeof(unsigned long long), s));
  CK(cudaMemsetAsync(err, 0, sizeof(unsigned int), s));

  DirectPass p{};
  p.inst = d_tab;
  p.ninst = K;
  p.no[0] = tab[0].side[0].no;
  p.no[1] = tab[0].side[1].no;
  p.class_bits = static_cast<uint32_t>(dp.B);
  p.cmask = cmask;
  p.insert_cap = (5u << dp.TB) / 8;  // about 5 of the 8 slots of a bucket
  p.match_key = match_key;
  p.match_cls = match_cls;
  p.match_count = match_count;
  p.match_cap = kDirectMatchCap;
  p.records = records;
  p.error = err;
  // launches of about 2^32 records (15 ms) and at most 2^20 classes in all:
  // a bounded kernel time, so cancellation (checked between launches) and
  // the kernels of other requests on higher-priority streams get their turn
  const uint32_t ncls = c_end - c_begin;
  const double rec_per_class = std::ldexp(1.0, dp.cols[0] - dp.B) + std::ldexp(1.0, dp.cols[1] - dp.B);
  const uint32_t per_launch = static_cast<uint32_t>(std::max<double>(
      1.0, std::min<double>(std::ldexp(1.0, 32) / rec_per_class, (double)(1u << 20)) / K));
  const uint32_t nlaunch = (ncls + per_launch - 1) / per_launch;
  CK(da.get(&work, nlaunch));
  CK(cudaMemsetAsync(work, 0, sizeof(unsigned int) * nlaunch, s));
  const double per_class_in = 4.0 * (p.no[0] + p.no[1]);
  int passes = 0;
  for (uint32_t li = 0; li < nlaunch; ++li) {
    if (cancel && *cancel) return fail(MSP_ECANCELED, "request canceled");
    p.c0 = c_begin + li * per_launch;
    p.nclass = std::min(per_launch, c_end - p.c0);
    p.work = work + li;
    // algorithmic bytes: 4 per record (its inner key) plus one bucket offset
    // per outer subset and class; the exact record count replaces this
    // estimate once the solve ends
    const double rec_est = (double)K * p.nclass * rec_per_class;
    LAUNCH(MSP_K_DIRECT, 1, static_cast<uint64_t>(4.0 * rec_est + per_class_in * p.nclass * K),
           launch_direct_join(dp.TB, p, s));
    ++passes;
  }
  unsigned long long nmatch = 0, nrec = 0;
  unsigned int err_h = 0;
  CK(cp.d2h(&nmatch, match_count, sizeof(nmatch)));
  CK(cp.d2h(&nrec, records, sizeof(nrec)));
  CK(cp.d2h(&err_h, err, sizeof(err_h)));
  CK(cudaStreamSynchronize(s));
  prof.flush();
  if (st) {
    st->passes = passes;
    st->records_done = nrec;
    st->key_matches = nmatch;
    if (prof.on) st->kernel_bytes[MSP_K_DIRECT] = 4 * nrec + static_cast<uint64_t>(per_class_in * ncls * K);
  }
  if (err_h || nmatch > kDirectMatchCap) return kDirectFallback;
  if (nmatch == 0) return MSP_OK;

  DirectVerify v{};
  v.inst = d_vtab;
  for (int sd = 0; sd < 2; ++sd) {
    v.qi[sd] = dp.qi[sd];
    v.col_o[sd] = dp.col_o[sd];
    v.col_i[sd] = dp.col_i[sd];
  }
  v.W = dp.W;
  v.class_bits = static_cast<uint32_t>(dp.B);
  v.cmask = cmask;
  v.match_key = match_key;
  v.match_cls = match_cls;
  unsigned long long *cnts;
  unsigned int *ovf;
  CK(da.get(&cnts, 2));
  CK(da.get(&ovf, 1));
  v.sol_count = cnts;
  v.pairs = cnts + 1;
  v.overflow = ovf;
  uint64_t cap = 1u << 16;
  for (int attempt = 0; attempt < 2; ++attempt) {
    uint64_t *sol;
    CK(da.get(&sol, 3 * cap));
    v.sol = sol;
    v.sol_cap = cap;
    CK(cudaMemsetAsync(cnts, 0, 2 * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(ovf, 0, sizeof(unsigned int), s));
    LAUNCH(MSP_K_VERIFY, 1, 0,
           (direct_verify_kernel<<<static_cast<unsigned>(nmatch), kVT, 0, s>>>(v), cudaGetLastError()));
    unsigned long long hc[2];
    unsigned int ovf_h = 0;
    CK(cp.d2h(hc, cnts, sizeof(hc)));
    CK(cp.d2h(&ovf_h, ovf, sizeof(ovf_h)));
    CK(cudaStreamSynchronize(s));
    if (ovf_h) return kDirectFallback;
    if (st) st->pairs_verified = hc[1];
    if (hc[0] <= cap) {
      std::vector<uint64_t> h(3 * hc[0]);
      if (hc[0]) {
        CK(cp.d2h(h.data(), sol, sizeof(uint64_t) * 3 * hc[0]));
        CK(cudaStreamSynchronize(s));
      }
      for (uint64_t i = 0; i < hc[0]; ++i) {
        const uint64_t k = h[3 * i + 2];
        if (k >= K) return fail(MSP_ECUDA, "verification produced an invalid instance tag");
        out[k].push_back(h[3 * i]);
        out[k].push_back(h[3 * i + 1]);
      }
      break;
    }
    if (hc[0] > (1ull << 28)) return fail(MSP_EOVERFLOW, "more than 2^28 solutions");
    cap = hc[0];
  }
  return MSP_OK;
}

}  // namespace

// Solves `inst` on the direct pass.  Returns MSP_OK with res (unsorted
// two-word masks), kDirectFallback when another path must solve it (out of
// memory for the inner lists, a class beyond the kernel's bounds, a match
// list or candidate list overflow), or an error status.
int solve_direct(msp_instance *inst, const DirectPlan &dp, const Plan &kp, size_t budget, Prof &prof,
                 std::vector<uint64_t> &res) {
  const int n = inst->n;
  msp_stats &st = inst->stats;
  cudaStream_t s = inst->stream;
  const uint32_t M = 1u << dp.B;
  if (direct_footprint(dp) > budget) return kDirectFallback;
  if (inst->part >= inst->parts) return fail(MSP_EINVAL, "class part must be below the number of parts");

  st.quarter[0] = dp.qo[0];
  st.quarter[1] = dp.qo[1];
  st.quarter[2] = dp.qi[0];
  st.quarter[3] = dp.qi[1];
  st.class_bits = dp.B;
  st.class_rows = dp.t;
  st.digit_bits = 0;

  DevAlloc da(s);
  Copier cp{&st, s};
  std::vector<DirectLists> lists(1);
  {
    uint32_t *cnt, *scantmp;
    CK(da.get(&cnt, (size_t)M + 1));
    CK(da.get(&scantmp, ((size_t)M + 1 + 4095) / 4096 + 1));
    const int rc = build_direct_lists(inst->A.data(), inst->d.data(), inst->m, n, dp, kp, da, cp, prof, cnt,
                                      scantmp, lists[0]);
    if (rc != MSP_OK) return rc;
    da.free1(cnt, sizeof(uint32_t) * ((size_t)M + 1));
  }

  // ---- C1: row-1 candidate pairs (the metric's unit of work) ----
  {
    int32_t *d_a1;
    unsigned __int128 *d_dp;
    unsigned long long *d_c1;
    const int d1 = inst->d[0];
    CK(da.get(&d_a1, n));
    CK(da.get(&d_dp, 2 * ((size_t)d1 + 1)));
    CK(da.get(&d_c1, 2));
    CK(cp.h2d(d_a1, inst->A.data(), sizeof(int32_t) * n));
    LAUNCH(MSP_K_C1, 1, 0, (c1_dp_kernel<<<1, 1024, 0, s>>>(d_a1, n, d1, d_dp, d_c1), cudaGetLastError()));
    unsigned long long c1h[2];
    CK(cp.d2h(c1h, d_c1, sizeof(c1h)));
    CK(cudaStreamSynchronize(s));
    st.row1_candidates_lo = c1h[0];
    st.row1_candidates_hi = c1h[1];
  }

  const uint32_t c_begin = static_cast<uint32_t>((uint64_t)M * inst->part / inst->parts);
  const uint32_t c_end = static_cast<uint32_t>((uint64_t)M * (inst->part + 1) / inst->parts);
  st.classes_total = M;
  st.classes_done = c_end - c_begin;
  std::vector<std::vector<uint64_t>> out;
  const int rc = run_direct(lists, dp, c_begin, c_end, da, cp, prof, &st, inst->cancel, out);
  if (rc != MSP_OK) return rc;
  res = std::move(out[0]);
  st.device_bytes = da.peak;
  da.release();
  CK(cudaStreamSynchronize(s));
  prof.flush();
  return MSP_OK;
}

// msp_solve_batch on the direct pass: every instance's lists, then one join
// launch (per 2^20 classes) over the classes of all instances and one
// verification launch over all matches.  raw[k]: unsorted two-word masks of
// instance k.  Returns MSP_OK, kDirectFallback or an error status.
int solve_batch_direct(const int32_t *const *A, const int32_t *const *d, int m, int n, int count,
                       std::vector<std::vector<uint64_t>> &raw, cudaStream_t s, size_t budget) {
  raw.assign(count, {});
  const DirectPlan dp = make_direct_plan(m, n, -1);
  if (!dp.ok) return kDirectFallback;
  const Plan kp = make_plan(m, n);
  const uint32_t M = 1u << dp.B;
  // feasible right-hand sides only
  std::vector<int> idx;
  for (int k = 0; k < count; ++k) {
    bool feasible = true;
    for (int i = 0; i < m && feasible; ++i) {
      int64_t rs = 0;
      for (int j = 0; j < n; ++j) rs += A[k][(size_t)i * n + j];
      feasible = d[k][i] <= rs;
    }
    if (feasible) idx.push_back(k);
  }
  const uint32_t K = static_cast<uint32_t>(idx.size());
  if (K == 0) return MSP_OK;
  // tags instance << B | class must fit 32 bits; lists of all instances
  // must fit the budget
  if ((uint64_t)K << dp.B > (1ull << 32)) return kDirectFallback;
  const double per_inst = 8.0 * (std::ldexp(1.0, dp.qi[0]) + std::ldexp(1.0, dp.qi[1])) +
                          16.0 * (std::ldexp(1.0, dp.B) + 1) + (64 << 10);
  if (per_inst * K + (double)direct_footprint(dp) > (double)budget) return kDirectFallback;

  DevAlloc da(s);
  Copier cp{nullptr, s};
  msp_stats scratch{};
  Prof prof;
  prof.s = s;
  prof.st = &scratch;
  std::vector<DirectLists> lists;
  {
    const int rc = build_direct_lists_batch(A, d, idx, m, n, dp, kp, da, cp, prof, lists);
    if (rc != MSP_OK) return rc;
  }
  std::vector<std::vector<uint64_t>> out;
  const int rc = run_direct(lists, dp, 0, M, da, cp, prof, nullptr, nullptr, out);
  if (rc != MSP_OK) return rc;
  for (uint32_t k = 0; k < K; ++k) raw[idx[k]] = std::move(out[k]);
  da.release();
  CK(cudaStreamSynchronize(s));
  return MSP_OK;
}

}  // namespace msp
