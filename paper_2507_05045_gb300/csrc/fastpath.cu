// Streaming pass of libmsp (sm_103a): the records of a residue pass are
// generated once, radix-partitioned through a thread-block cluster, and
// joined by a persistent kernel fed with bulk asynchronous copies.
//
//   class_size_kernel   exact class sizes |L_r| = sum_u |Q1[u]| |Q3[r-u]|
//                       (cyclic convolution of the bucket histograms).
//   scatter_fast_kernel per cluster round every block generates up to 8192
//                       records into registers and ranks them by the top D
//                       key bits in shared memory; the blocks of the cluster
//                       exchange their digit histograms through distributed
//                       shared memory, one owner block per digit reserves
//                       the cluster's run with a single global atomic, and
//                       every block writes its part of the run, so a digit's
//                       records leave the cluster as one contiguous run.
//                       Partitions have a fixed capacity (mean + 8 sigma);
//                       a record past it raises the pass's overflow flag and
//                       the host re-runs that pass on the exact path.
//   join_fast_kernel    persistent: while a partition is sorted and joined
//                       in shared memory, the next one is already streaming
//                       in by cp.async.bulk (1-D TMA) on an mbarrier.
#include "msp_internal.cuh"

#include <cooperative_groups.h>

#include <algorithm>

namespace cg = cooperative_groups;

namespace msp {

namespace {

__device__ __forceinline__ uint32_t lane() { return threadIdx.x & 31; }

// Compile-time digit widths: the top D bits and the next S bits of a key,
// both inside its high 32-bit word (D + S <= 32).
template <int D>
__device__ __forceinline__ uint32_t digit_t(uint64_t key) {
  if constexpr (D == 0) {
    return 0u;
  } else {
    return static_cast<uint32_t>(key >> 32) >> (32 - D);
  }
}

template <int D, int S>
__device__ __forceinline__ uint32_t subkey_t(uint64_t key) {
  static_assert(D + S <= 32, "digit and sub-key must fit the high word");
  return (static_cast<uint32_t>(key >> 32) >> (32 - D - S)) & ((1u << S) - 1u);
}

template <typename T>
__device__ T scan_excl(T v, T *wt, T *total) {
  const int ln = lane(), wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (ln >= o) x += y;
  }
  if (ln == 31) wt[wp] = x;
  __syncthreads();
  if (wp == 0) {
    T t = ln < nw ? wt[ln] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, t, o);
      if (ln >= o) t += y;
    }
    if (ln < nw) wt[ln] = t;
  }
  __syncthreads();
  const T before = wp ? wt[wp - 1] : T(0);
  *total = wt[nw - 1];
  __syncthreads();
  return x + before - v;
}

// Exclusive scan of a shared array of n entries in place.  Warp w scans the
// contiguous chunk [w*n/W, (w+1)*n/W) 32 entries at a time with shuffles;
// the warp totals are scanned by warp 0 and added back.  *total = sum.
__device__ void scan_array(uint32_t *a, int n, uint32_t *wt, uint32_t *total) {
  const int ln = lane(), wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int per = (n + nw - 1) / nw;
  const int b0 = min(wp * per, n), b1 = min(b0 + per, n);
  uint32_t carry = 0;
  for (int c = b0; c < b1; c += 32) {
    const int i = c + ln;
    const uint32_t v = i < b1 ? a[i] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (ln >= o) x += y;
    }
    if (i < b1) a[i] = carry + x - v;
    carry += __shfl_sync(0xffffffffu, x, 31);
  }
  if (ln == 0) wt[wp] = carry;
  __syncthreads();
  if (wp == 0) {
    uint32_t t = ln < nw ? wt[ln] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (ln >= o) t += y;
    }
    if (ln < nw) wt[ln] = t;  // inclusive
  }
  __syncthreads();
  const uint32_t before = wp ? wt[wp - 1] : 0u;
  if (before)
    for (int i = b0 + ln; i < b1; i += 32) a[i] += before;
  *total = wt[nw - 1];
  __syncthreads();
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst_smem)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

}  // namespace

// -------------------------------------------------------------------------
// Exact class sizes: out[r] = sum_u n_O[u] * n_I[(r - u) mod M].
// A block owns kCsR consecutive r and walks u in tiles: the tile of n_O and
// the window of n_I it needs are staged in shared memory.
// -------------------------------------------------------------------------
constexpr int kCsR = 256;
constexpr int kCsU = 1024;

__global__ void __launch_bounds__(kCsR) class_size_kernel(const uint32_t *__restrict__ offO,
                                                          const uint32_t *__restrict__ offI, uint32_t M,
                                                          uint32_t rbeg, uint32_t rcount,
                                                          unsigned long long *out) {
  __shared__ uint32_t sO[kCsU];
  __shared__ uint32_t sI[kCsU + kCsR];
  const uint32_t r0 = rbeg + blockIdx.x * kCsR;  // classes of this block: [r0, r0 + kCsR)
  const uint32_t ri = blockIdx.x * kCsR + threadIdx.x;
  const uint32_t r = r0 + threadIdx.x;
  const uint32_t mask = M - 1u;
  unsigned long long acc = 0;
  for (uint32_t u0 = 0; u0 < M; u0 += kCsU) {
    const uint32_t nu = min(static_cast<uint32_t>(kCsU), M - u0);
    for (uint32_t i = threadIdx.x; i < nu; i += blockDim.x) sO[i] = offO[u0 + i + 1] - offO[u0 + i];
    // n_I[(r - u) mod M] for r in [r0, r0+kCsR), u in [u0, u0+nu):
    // index w = r0 - u0 - (nu - 1) + k, k in [0, nu - 1 + kCsR)
    const uint32_t wbase = (r0 - u0 - (nu - 1)) & mask;
    for (uint32_t k = threadIdx.x; k < nu - 1 + kCsR; k += blockDim.x) {
      const uint32_t w = (wbase + k) & mask;
      sI[k] = offI[w + 1] - offI[w];
    }
    __syncthreads();
    if (ri < rcount) {
      // u = u0 + i  ->  k = (r - r0) + (nu - 1) - i
      const uint32_t kb = threadIdx.x + (nu - 1);
      for (uint32_t i = 0; i < nu; ++i) acc += static_cast<unsigned long long>(sO[i]) * sI[kb - i];
    }
    __syncthreads();
  }
  if (ri < rcount) out[ri] = acc;
  (void)r;
}

cudaError_t launch_class_sizes(const uint32_t *offO, const uint32_t *offI, uint32_t M, uint32_t rbeg,
                               uint32_t rcount, unsigned long long *out, cudaStream_t s) {
  if (rcount == 0) return cudaSuccess;
  const uint32_t blocks = (rcount + kCsR - 1) / kCsR;
  class_size_kernel<<<blocks, kCsR, 0, s>>>(offO, offI, M, rbeg, rcount, out);
  return cudaGetLastError();
}

// -------------------------------------------------------------------------
// Scatter (S3 + the first radix digit of S4).
// A block owns a slice of one class (side, class, outer range) and walks it
// in rounds of up to kScRound records.  Each round:
//   1. window: up to kScW outer elements, their inner buckets r - kappa(o),
//      and a block scan of the bucket sizes; empty buckets are compacted out,
//      so the record prefix over the window is strictly increasing;
//   2. generation: warp w takes records [w*512, w*512 + 512) in 16 batches
//      of 32 consecutive records.  The lane of record K + lane finds its
//      outer element without branching: the starts of the next 32 elements
//      that fall inside the batch are OR-reduced into a 32-bit mask and the
//      element is e0 + popcount(mask & lanes<=lane).  key = K(o) + K(i);
//   3. rank by the top D key bits (shared atomics), block scan of the digit
//      histogram, one global atomic per nonempty digit reserves this round's
//      run in the partition (class, digit);
//   4. records are placed by digit in shared memory and leave as contiguous
//      runs (one write burst per digit).
// Partitions have a fixed capacity; a record past it is dropped and the
// pass's overflow flag raised (the host re-runs that pass on the exact path).
// -------------------------------------------------------------------------
constexpr int kScT = 256;                    // threads per block
constexpr int kScBatches = 16;               // batches of 32 records per warp and round
constexpr int kScRound = kScT * kScBatches;  // 4096 records per round
constexpr int kScE = 4;                      // outer elements per thread in a window
constexpr int kScW = kScT * kScE;            // 1024 outer elements per window

struct __align__(16) DigitDesc {
  unsigned long long dst;  // record index of sorted position 0 of this digit's run
  uint32_t lim;            // sorted positions below lim are inside the partition
  uint32_t pad;
};

size_t scatter_fast_smem(int D) {
  const size_t nd = size_t(1) << D;
  return kScRound * sizeof(uint64_t)         // records placed by digit
         + kScW * sizeof(uint64_t)           // outer keys of the window
         + nd * sizeof(DigitDesc)            // per-digit destinations
         + kScW * sizeof(uint32_t)           // inner bucket starts
         + (kScW + 1) * sizeof(uint32_t)     // record prefix of the window
         + 2 * nd * sizeof(uint32_t)         // histogram, local offsets
         + kScW * sizeof(uint16_t)           // window index of each nonempty element
         + 64;
}

template <int D>
__global__ void __launch_bounds__(kScT, 3) scatter_fast_kernel(FastPass p, int nwu) {
  extern __shared__ __align__(16) uint8_t sm[];
  constexpr int nd = 1 << D;
  uint64_t *sorted = reinterpret_cast<uint64_t *>(sm);
  uint64_t *s_ko = sorted + kScRound;
  DigitDesc *desc = reinterpret_cast<DigitDesc *>(s_ko + kScW);
  uint32_t *s_ib = reinterpret_cast<uint32_t *>(desc + nd);
  uint32_t *s_pre = s_ib + kScW;
  uint32_t *hist = s_pre + kScW + 1;
  uint32_t *loff = hist + nd;
  uint16_t *s_orig = reinterpret_cast<uint16_t *>(loff + nd);
  __shared__ unsigned long long s_wt64[32];
  __shared__ uint32_t s_wt[32];

  const int lanei = static_cast<int>(lane());
  const int warp = threadIdx.x >> 5;
  for (int wu = blockIdx.x; wu < nwu; wu += gridDim.x) {
    int side, cl, sl;
    const int per_inst = p.nclass * (p.slices[0] + p.slices[1]);
    const int inst_i = wu / per_inst;
    const FastInst &fi = p.inst[inst_i];
    {
      const int nb0 = p.nclass * p.slices[0];
      int b = wu % per_inst;
      if (b < nb0) {
        side = 0;
      } else {
        side = 1;
        b -= nb0;
      }
      cl = b / p.slices[side];
      sl = b % p.slices[side];
    }
    const SideGen &g = fi.side[side];
    const uint64_t *__restrict__ okey = g.okey;
    const uint32_t *__restrict__ ocls = g.ocls;
    const uint64_t *__restrict__ ikey = g.ikey;
    const uint32_t *__restrict__ ioff = g.ioff;
    const int64_t osize = g.osize;
    const int64_t slice_outer = g.slice_outer;
    const int wmax = g.wmax;
    const uint32_t cg_id = static_cast<uint32_t>(p.c0 + cl);
    const uint32_t r = cg_id & p.cmask;
    const int64_t o_end = min((int64_t)(sl + 1) * slice_outer, osize);
    int64_t o_cur = (int64_t)sl * slice_outer;
    uint32_t j_cur = 0;
    const uint32_t cap = fi.cap[side][cg_id];
    const unsigned long long seg0 = fi.class_base[side][cg_id];
    uint64_t *const rec = p.rec[side];
    uint32_t *const fill = fi.fill[side] + (int64_t)cl * nd;

    while (o_cur < o_end) {
      // ---- 1. window ----
      const int w_n = static_cast<int>(min(static_cast<int64_t>(wmax), o_end - o_cur));
      uint32_t cnt[kScE], ibv[kScE];
      uint64_t kov[kScE];
      unsigned long long recs = 0;
      uint32_t nonempty = 0;
#pragma unroll
      for (int e = 0; e < kScE; ++e) {
        const int idx = threadIdx.x * kScE + e;
        cnt[e] = 0;
        if (idx < w_n) {
          const int64_t o = o_cur + idx;
          const uint32_t w = (r - ocls[o]) & p.cmask;
          uint32_t ib = ioff[w];
          uint32_t c = ioff[w + 1] - ib;
          if (idx == 0) {
            ib += j_cur;
            c -= j_cur;
          }
          cnt[e] = c;
          ibv[e] = ib;
          kov[e] = okey[o];
          recs += c;
          nonempty += c ? 1u : 0u;
        }
      }
      for (int i = threadIdx.x; i < nd; i += kScT) hist[i] = 0;
      unsigned long long tot_packed;
      // low 12 bits: nonempty elements (< 4096), high bits: records
      const unsigned long long ex =
          scan_excl<unsigned long long>((recs << 12) | nonempty, s_wt64, &tot_packed);
      {
        uint32_t pos = static_cast<uint32_t>(ex & 0xfffu);
        unsigned long long pre = ex >> 12;
#pragma unroll
        for (int e = 0; e < kScE; ++e) {
          if (cnt[e]) {
            s_ko[pos] = kov[e];
            s_ib[pos] = ibv[e];
            s_pre[pos] = static_cast<uint32_t>(min(pre, 0xffffffffull));
            s_orig[pos] = static_cast<uint16_t>(threadIdx.x * kScE + e);
            ++pos;
            pre += cnt[e];
          }
        }
      }
      const uint32_t nne = static_cast<uint32_t>(tot_packed & 0xfffu);
      const unsigned long long total = tot_packed >> 12;
      if (threadIdx.x == 0) s_pre[nne] = static_cast<uint32_t>(min(total, 0xffffffffull));
      __syncthreads();
      const uint32_t n_round = static_cast<uint32_t>(min(static_cast<unsigned long long>(kScRound), total));

      // ---- 2. generation: 16 batches of 32 consecutive records per warp ----
      uint64_t keys[kScBatches];
      uint32_t rank[kScBatches];
      const uint32_t K0 = static_cast<uint32_t>(warp) * (kScBatches * 32);
      if (K0 < n_round) {
        uint32_t lo = 0, hi = nne - 1;  // last element whose prefix is <= K0
        while (lo < hi) {
          const uint32_t mid = (lo + hi + 1) >> 1;
          if (s_pre[mid] <= K0) lo = mid; else hi = mid - 1;
        }
        uint32_t e0 = lo;             // element holding record K of the batch
        uint32_t st0 = s_pre[lo];     // its first record
        const uint32_t lemask = (2u << lanei) - 1u;  // lanes <= this lane
#pragma unroll
        for (int b = 0; b < kScBatches; ++b) {
          const uint32_t K = K0 + b * 32;
          if (K < n_round) {  // warp-uniform
            const uint32_t t = e0 + 1 + lanei;
            const uint32_t P = t <= nne ? s_pre[t] : 0xffffffffu;
            const uint32_t off = P - K;  // >= 1: element e0 holds record K
            const unsigned mask = __reduce_or_sync(0xffffffffu, off < 32u ? (1u << off) : 0u);
            const uint32_t c = __popc(mask & lemask);
            const uint32_t shp = __shfl_sync(0xffffffffu, P, (c - 1u) & 31u);
            const uint32_t e = e0 + c;
            const uint32_t start = c ? shp : st0;
            const uint32_t k = K + lanei;
            if (k < n_round) {
              const uint64_t key = s_ko[e] + ikey[s_ib[e] + (k - start)];
              keys[b] = key;
              rank[b] = atomicAdd(&hist[digit_t<D>(key)], 1u);
            }
            e0 = __shfl_sync(0xffffffffu, e, 31);
            st0 = __shfl_sync(0xffffffffu, start, 31);
          }
        }
      }
      __syncthreads();
      // ---- advance the cursor past this round's records ----
      if (n_round == total) {
        o_cur += w_n;
        j_cur = 0;
      } else {
        uint32_t lo = 0, hi = nne - 1;
        while (lo < hi) {
          const uint32_t mid = (lo + hi + 1) >> 1;
          if (s_pre[mid] <= n_round) lo = mid; else hi = mid - 1;
        }
        const uint32_t oi = s_orig[lo];
        j_cur = (n_round - s_pre[lo]) + (oi == 0 ? j_cur : 0u);
        o_cur += oi;
      }
      // ---- 3. digit offsets and one reservation per nonempty digit ----
      for (int i = threadIdx.x; i < nd; i += kScT) loff[i] = hist[i];
      __syncthreads();
      uint32_t tot2;
      scan_array(loff, nd, s_wt, &tot2);
      bool ovf = false;
      for (int gd = threadIdx.x; gd < nd; gd += kScT) {
        const uint32_t h = hist[gd];
        if (h) {
          const uint32_t base = atomicAdd(fill + gd, h);
          const uint32_t fit = base < cap ? min(h, cap - base) : 0u;
          ovf |= fit < h;
          DigitDesc dd;
          dd.dst = seg0 + (unsigned long long)gd * cap + base - loff[gd];
          dd.lim = loff[gd] + fit;
          dd.pad = 0;
          desc[gd] = dd;
        }
      }
      if (ovf) atomicOr(p.overflow + inst_i, 1u);
      // ---- 4. place by digit, then write the runs ----
      if (K0 < n_round) {
#pragma unroll
        for (int b = 0; b < kScBatches; ++b) {
          const uint32_t k = K0 + b * 32 + lanei;
          if (k < n_round) sorted[loff[digit_t<D>(keys[b])] + rank[b]] = keys[b];
        }
      }
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < n_round; i += kScT) {
        const uint64_t key = sorted[i];
        const DigitDesc dd = desc[digit_t<D>(key)];
        if (i < dd.lim) rec[dd.dst + i] = key;
      }
      __syncthreads();
    }
  }
}

template <int D>
static cudaError_t launch_scatter_d(const FastPass &p, int nclass_run, cudaStream_t s) {
  static size_t attr = 0;
  static int per_sm = 0;
  static int sms = 0;
  const size_t smem = scatter_fast_smem(D);
  if (smem > attr) {
    cudaError_t e = cudaFuncSetAttribute(scatter_fast_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    attr = smem;
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, scatter_fast_kernel<D>, kScT, smem) != cudaSuccess ||
        n < 1) {
      cudaGetLastError();
      n = 1;
    }
    per_sm = n;
  }
  FastPass q = p;
  q.nclass = nclass_run;
  const int nwu = p.ninst * nclass_run * (p.slices[0] + p.slices[1]);
  const int blocks = std::max(1, std::min(nwu, per_sm * sms));
  scatter_fast_kernel<D><<<blocks, kScT, smem, s>>>(q, nwu);
  return cudaGetLastError();
}

cudaError_t launch_scatter_fast(const FastPass &p, int nclass_run, cudaStream_t s) {
  switch (p.D) {
    case 0: return launch_scatter_d<0>(p, nclass_run, s);
    case 1: return launch_scatter_d<1>(p, nclass_run, s);
    case 2: return launch_scatter_d<2>(p, nclass_run, s);
    case 3: return launch_scatter_d<3>(p, nclass_run, s);
    case 4: return launch_scatter_d<4>(p, nclass_run, s);
    case 5: return launch_scatter_d<5>(p, nclass_run, s);
    case 6: return launch_scatter_d<6>(p, nclass_run, s);
    case 7: return launch_scatter_d<7>(p, nclass_run, s);
    case 8: return launch_scatter_d<8>(p, nclass_run, s);
    case 9: return launch_scatter_d<9>(p, nclass_run, s);
    case 10: return launch_scatter_d<10>(p, nclass_run, s);
    case 11: return launch_scatter_d<11>(p, nclass_run, s);
    case 12: return launch_scatter_d<12>(p, nclass_run, s);
    default: return cudaErrorInvalidValue;
  }
}

// -------------------------------------------------------------------------
// Join (S4 second digit + S5).  Persistent, one block of 1024 threads per SM.
// Partition s = (class, digit): the left keys arrive by cp.async.bulk into
// one of two buffers (the next partition's left side streams in while this
// one is processed), the right keys into a third buffer.  The left side is
// counting-sorted in place by the next S key bits; every right key probes
// its bucket.  The first left element equal to the key is claimed with a
// shared bit (so duplicate right keys emit once) and the (class, key) pair
// is appended with one atomic per warp.
// -------------------------------------------------------------------------
constexpr int kJT = 1024;
constexpr int kJReg = (kFastCap + kJT - 1) / kJT;

size_t join_fast_smem(int S) {
  return 3 * (size_t)kFastCap * sizeof(uint64_t) + (((size_t)1 << S) + 1) * sizeof(uint32_t) +
         (kFastCap / 32 + 1) * sizeof(uint32_t) + 64;
}

struct SegRef {
  const uint64_t *L, *R;
  uint32_t nL, nR;
  uint32_t cls;  // tag + class id of the partition
};

__device__ __forceinline__ SegRef seg_ref(const FastPass &p, int s) {
  const int nd = 1 << p.D;
  const int per_inst = p.nclass << p.D;
  const FastInst &fi = p.inst[s / per_inst];
  const int rem = s % per_inst;
  const int cl = rem >> p.D, gd = rem & (nd - 1);
  const uint32_t cg_id = static_cast<uint32_t>(p.c0 + cl);
  SegRef r;
  const uint32_t capL = fi.cap[0][cg_id], capR = fi.cap[1][cg_id];
  r.L = p.rec[0] + fi.class_base[0][cg_id] + (uint64_t)gd * capL;
  r.R = p.rec[1] + fi.class_base[1][cg_id] + (uint64_t)gd * capR;
  r.nL = min(fi.fill[0][(int64_t)cl * nd + gd], capL);
  r.nR = min(fi.fill[1][(int64_t)cl * nd + gd], capR);
  if (r.nL == 0 || r.nR == 0) r.nL = r.nR = 0;
  r.cls = fi.tag + (cg_id & p.cmask);
  return r;
}

// One bulk copy of n keys (rounded up to 16 bytes; partitions are 16-record
// multiples, so the rounding stays inside the partition) on `bar`.
__device__ __forceinline__ void issue_keys(const uint64_t *src, uint32_t n, uint64_t *dst, uint64_t *bar) {
  const uint32_t bytes = ((n + 1u) & ~1u) * 8u;
  mbar_arrive_expect_tx(bar, bytes);
  if (bytes) bulk_load(dst, src, bytes, bar);
}

// Bounded wait on an mbarrier phase: thread 0 waits (2 s limit, then sets
// the error flag and waits once more, bounded), the block learns the outcome
// through shared memory, then every thread observes the completed phase.
__device__ __forceinline__ bool wait_phase(uint64_t *bar, uint32_t parity, unsigned int *err, int *s_ok) {
  if (threadIdx.x == 0) {
    const uint64_t t0 = global_ns();
    bool ok = true;
    while (!mbar_try_wait(bar, parity)) {
      if (global_ns() - t0 > 2000000000ull) {
        ok = false;
        break;
      }
    }
    if (!ok) {
      atomicOr(err, 1u);
      const uint64_t t1 = global_ns();
      while (!mbar_try_wait(bar, parity) && global_ns() - t1 < 2000000000ull) {
      }
    }
    *s_ok = ok ? 1 : 0;
  }
  __syncthreads();
  if (!*s_ok) return false;
  while (!mbar_try_wait(bar, parity)) {
  }
  return true;
}

template <int D, int S>
__device__ void sort_in_place(uint64_t *buf, uint32_t n, uint32_t *off, uint32_t *wt) {
  constexpr int nb = 1 << S;
  uint64_t k[kJReg];
  uint32_t rk[kJReg];
#pragma unroll
  for (int q = 0; q < kJReg; ++q) {
    const uint32_t i = threadIdx.x + q * kJT;
    if (i < n) {
      k[q] = buf[i];
      rk[q] = atomicAdd(&off[subkey_t<D, S>(k[q])], 1u);
    }
  }
  __syncthreads();
  uint32_t tot;
  scan_array(off, nb, wt, &tot);
  if (threadIdx.x == 0) off[nb] = tot;
#pragma unroll
  for (int q = 0; q < kJReg; ++q) {
    const uint32_t i = threadIdx.x + q * kJT;
    if (i < n) buf[off[subkey_t<D, S>(k[q])] + rk[q]] = k[q];
  }
}

__device__ __forceinline__ void emit(const FastPass &p, bool e, uint64_t key, uint32_t cls) {
  const unsigned bal = __ballot_sync(0xffffffffu, e);
  if (!bal) return;
  const int leader = __ffs(bal) - 1;
  unsigned long long base = 0;
  if (static_cast<int>(lane()) == leader) base = atomicAdd(p.match_count, (unsigned long long)__popc(bal));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (e) {
    const unsigned long long slot = base + __popc(bal & ((1u << lane()) - 1u));
    if (slot < p.match_cap) {
      p.match_key[slot] = key;
      p.match_cls[slot] = cls;
    }
  }
}

constexpr int kJS = 11;  // sub-key bits of the in-partition sort

template <int D>
__global__ void __launch_bounds__(kJT, 1) join_fast_kernel(FastPass p, int nseg) {
  extern __shared__ __align__(16) uint8_t sm[];
  uint64_t *const bufL0 = reinterpret_cast<uint64_t *>(sm);  // two left buffers
  uint64_t *const bufR = bufL0 + 2 * kFastCap;
  constexpr int S = kJS;
  constexpr int nb = 1 << S;
  uint32_t *off = reinterpret_cast<uint32_t *>(bufR + kFastCap);
  uint32_t *flags = off + nb + 1;
  const int nflag = kFastCap / 32 + 1;
  __shared__ __align__(8) uint64_t barL[2];
  __shared__ __align__(8) uint64_t barR;
  __shared__ uint32_t s_wt[32];
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    mbar_init(&barL[0], 1);
    mbar_init(&barL[1], 1);
    mbar_init(&barR, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int G = gridDim.x;
  int s = blockIdx.x;
  if (s < nseg && threadIdx.x == 0) {
    const SegRef r0 = seg_ref(p, s);
    issue_keys(r0.L, r0.nL, bufL0, &barL[0]);
    issue_keys(r0.R, r0.nR, bufR, &barR);
  }
  uint32_t phL = 0, phR = 0;  // bit st of phL: parity of left buffer st
  for (int k = 0; s < nseg; ++k, s += G) {
    const int st = k & 1;
    const SegRef r = seg_ref(p, s);
    const int sn = s + G;
    if (sn < nseg && threadIdx.x == 0) {
      fence_proxy_async();
      const SegRef rn = seg_ref(p, sn);
      issue_keys(rn.L, rn.nL, bufL0 + (st ^ 1) * kFastCap, st ? &barL[0] : &barL[1]);
    }
    for (int i = threadIdx.x; i <= nb; i += kJT) off[i] = 0;
    for (int i = threadIdx.x; i < nflag; i += kJT) flags[i] = 0;
    if (!wait_phase(st ? &barL[1] : &barL[0], (phL >> st) & 1u, p.error, &s_ok)) return;
    phL ^= 1u << st;
    uint64_t *bL = bufL0 + st * kFastCap;
    if (r.nL) sort_in_place<D, S>(bL, r.nL, off, s_wt);
    if (!wait_phase(&barR, phR, p.error, &s_ok)) return;  // includes a block barrier
    phR ^= 1u;
    if (r.nR) {
      const uint32_t cls = r.cls;
      const uint32_t rounds = (r.nR + kJT - 1) / kJT;
      for (uint32_t rd = 0; rd < rounds; ++rd) {
        const uint32_t i = rd * kJT + threadIdx.x;
        bool e = false;
        uint64_t key = 0;
        if (i < r.nR) {
          key = bufR[i];
          const uint32_t b = subkey_t<D, S>(key);
          const uint32_t je = off[b + 1];
          for (uint32_t j = off[b]; j < je; ++j) {
            if (bL[j] == key) {
              const uint32_t bit = 1u << (j & 31);
              e = (atomicOr(&flags[j >> 5], bit) & bit) == 0;
              break;
            }
          }
        }
        emit(p, e, key, cls);
      }
    }
    __syncthreads();
    if (sn < nseg && threadIdx.x == 0) {
      fence_proxy_async();
      const SegRef rn = seg_ref(p, sn);
      issue_keys(rn.R, rn.nR, bufR, &barR);
    }
  }
}

template <int D>
static cudaError_t launch_join_d(const FastPass &p, int nclass_run, cudaStream_t s) {
  static size_t attr = 0;
  static int sms = 0;
  const size_t smem = join_fast_smem(kJS);
  if (smem > attr) {
    cudaError_t e = cudaFuncSetAttribute(join_fast_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    attr = smem;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  FastPass q = p;
  q.nclass = nclass_run;
  const int nseg = p.ninst * (nclass_run << D);
  const int blocks = std::min(nseg, sms);
  if (blocks < 1) return cudaSuccess;
  join_fast_kernel<D><<<blocks, kJT, smem, s>>>(q, nseg);
  return cudaGetLastError();
}

cudaError_t launch_join_fast(const FastPass &p, int nclass_run, cudaStream_t s) {
  if (p.S != kJS) return cudaErrorInvalidValue;
  switch (p.D) {
    case 0: return launch_join_d<0>(p, nclass_run, s);
    case 1: return launch_join_d<1>(p, nclass_run, s);
    case 2: return launch_join_d<2>(p, nclass_run, s);
    case 3: return launch_join_d<3>(p, nclass_run, s);
    case 4: return launch_join_d<4>(p, nclass_run, s);
    case 5: return launch_join_d<5>(p, nclass_run, s);
    case 6: return launch_join_d<6>(p, nclass_run, s);
    case 7: return launch_join_d<7>(p, nclass_run, s);
    case 8: return launch_join_d<8>(p, nclass_run, s);
    case 9: return launch_join_d<9>(p, nclass_run, s);
    case 10: return launch_join_d<10>(p, nclass_run, s);
    case 11: return launch_join_d<11>(p, nclass_run, s);
    case 12: return launch_join_d<12>(p, nclass_run, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace msp
