// Streaming pass of libmsp (sm_103a): the records of a residue pass are
// generated once, radix-partitioned by the top D key bits into partitions of
// fixed capacity, and joined by a persistent kernel fed with bulk
// asynchronous copies.
//
//   class_size_kernel   exact class sizes |L_r| = sum_u |Q1[u]| |Q3[r-u]|
//                       (cyclic convolution of the bucket histograms).
//   scatter_fast_kernel per round a block generates 4096 records into
//                       registers, ranks them by digit in shared memory,
//                       reserves each digit's run with one global atomic and
//                       writes the runs contiguously.  A record past its
//                       partition's capacity raises the instance's overflow
//                       flag and the host re-runs that pass on the exact path.
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

// Compile-time digit width: the top D bits of a key.
template <int D>
__device__ __forceinline__ uint32_t digit_t(uint64_t key) {
  if constexpr (D == 0) {
    return 0u;
  } else {
    return static_cast<uint32_t>(key >> 32) >> (32 - D);
  }
}

// Block-wide exclusive scan of one value per thread; *total is the block's
// sum.  One block barrier: every warp scans the warp totals itself.  With
// reuse a second barrier follows, so that the next call may overwrite wt;
// a caller that passes a block barrier before its next call passes false.
template <typename T>
__device__ T scan_excl(T v, T *wt, T *total, bool reuse) {
  const int ln = lane(), wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (ln >= o) x += y;
  }
  if (ln == 31) wt[wp] = x;
  __syncthreads();
  T t = ln < nw ? wt[ln] : T(0);
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, t, o);
    if (ln >= o) t += y;
  }
  // wp is warp-uniform: every lane reads the same source lane
  const T b = __shfl_sync(0xffffffffu, t, wp > 0 ? wp - 1 : 0);
  *total = __shfl_sync(0xffffffffu, t, nw - 1);
  if (reuse) __syncthreads();
  return x + (wp > 0 ? b : T(0)) - v;
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

// The same sizes from the outer elements themselves, for an outer list of
// fewer elements than classes: out[r] = sum over elements e of
// n_I[(r - class(e)) mod M].  A block owns kCsR consecutive r (so a warp's
// bucket loads are contiguous) and walks the elements' classes in tiles
// staged in shared memory.  Work: elements x classes of the range.
constexpr int kCsE = 2048;

__global__ void __launch_bounds__(kCsR) class_size_elems_kernel(const uint32_t *__restrict__ ocls, int64_t no,
                                                                const uint32_t *__restrict__ offI, uint32_t M,
                                                                uint32_t rbeg, uint32_t rcount,
                                                                unsigned long long *out) {
  __shared__ uint32_t sc[kCsE];
  const uint32_t ri = blockIdx.x * kCsR + threadIdx.x;
  const uint32_t r = rbeg + ri;
  const uint32_t mask = M - 1u;
  unsigned long long acc = 0;
  for (int64_t e0 = 0; e0 < no; e0 += kCsE) {
    const int ne = static_cast<int>(min(static_cast<int64_t>(kCsE), no - e0));
    for (int i = threadIdx.x; i < ne; i += kCsR) sc[i] = ocls[e0 + i];
    __syncthreads();
    if (ri < rcount)
      for (int i = 0; i < ne; ++i) {
        const uint32_t w = (r - sc[i]) & mask;
        acc += offI[w + 1] - offI[w];
      }
    __syncthreads();
  }
  if (ri < rcount) out[ri] = acc;
}

cudaError_t launch_class_sizes_elems(const uint32_t *ocls, int64_t no, const uint32_t *offI, uint32_t M,
                                     uint32_t rbeg, uint32_t rcount, unsigned long long *out, cudaStream_t s) {
  if (rcount == 0) return cudaSuccess;
  const uint32_t blocks = (rcount + kCsR - 1) / kCsR;
  class_size_elems_kernel<<<blocks, kCsR, 0, s>>>(ocls, no, offI, M, rbeg, rcount, out);
  return cudaGetLastError();
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
//   1. window: up to wmax outer elements, their inner buckets r - kappa(o)
//      and a block scan of the bucket sizes.  Nonempty elements are
//      compacted: element e keeps its outer key and delta(e) = (first inner
//      index) - (first record of e in the round), so record k of the round
//      reads inner index delta(e) + k; a bitmap marks the record at which
//      each element starts;
//   2. generation: warp w owns records [256 w, 256 w + 256).  The element of
//      record k is (elements starting before the warp's range) + popcount of
//      the bitmap bits up to k, minus one; key = K(o) + K(i), ranked by its
//      top D bits with a shared-memory atomic; keys and ranks stay in
//      registers;
//   3. digit offsets by a block scan, one global atomic per nonempty digit
//      reserves the round's run in the partition (class, digit);
//   4. keys are placed by digit in shared memory (over the window arrays,
//      which are dead by then) and leave as contiguous runs.
// Partitions have a fixed capacity; a record past it is dropped and the
// instance's overflow flag raised (the host re-runs that pass on the exact
// path).
// -------------------------------------------------------------------------
constexpr int kScT = 512;                   // threads per block
constexpr int kScPer = 8;                   // records per thread and round
constexpr int kScRound = kScT * kScPer;     // 4096 records per round
constexpr int kScE = 4;                     // outer elements per thread in a window
constexpr int kScW = kScT * kScE;           // at most 2048 outer elements per window
constexpr int kScWords = kScRound / 32;     // bitmap words
static_assert(kScW <= kScRound, "compacted elements must fit the window arrays");

struct __align__(16) DigitDesc {
  uint64_t *dst;  // where sorted position 0 of this digit's run would go
  uint32_t lim;   // sorted positions below lim are inside the partition
  uint32_t pad;
};

int scatter_window(int64_t inner_size, uint32_t classes) {
  // outer elements whose inner buckets hold about one round of records
  const double avg = std::max(1.0 / 64, (double)inner_size / (double)std::max<uint32_t>(1, classes));
  const double w = (double)kScRound / avg;
  return static_cast<int>(std::min<double>(kScW, std::max<double>(32, w)));
}

size_t scatter_fast_smem(int D) {
  const size_t nd = size_t(1) << D;
  return (size_t)kScRound * (sizeof(uint64_t) + sizeof(uint32_t))  // outer keys + deltas / sorted keys
         + nd * sizeof(DigitDesc)                                   // per-digit destinations
         + 2 * nd * sizeof(uint32_t)                                // histogram, local offsets
         + kScWords * sizeof(uint32_t)                              // element-start bitmap
         + 64;
}

// Block-uniform state of the work unit being scattered.  It lives in shared
// memory and every phase re-reads what it needs after the block barrier, so
// the keys and ranks of a round, not loop invariants, hold the registers.
struct ScatterUnit {
  const uint64_t *okey;
  const uint32_t *ocls;
  const uint64_t *ikey;
  const uint32_t *ioff;
  int64_t isize;  // inner list entries (the bound of the MSP_CHECKED checks)
  uint64_t *rec;
  uint32_t *fill;
  unsigned long long seg0;
  long long o_cur, o_end;
  uint32_t j_cur, cap, r, wmax;
  int inst;
};

template <int D>
__global__ void __launch_bounds__(kScT, 1024 / kScT) scatter_fast_kernel(FastPass p, int nwu) {
  extern __shared__ __align__(16) uint8_t sm[];
  constexpr int nd = 1 << D;
  constexpr int pd = (nd + kScT - 1) / kScT;  // digits per thread in the digit phase
  uint64_t *const s_ko = reinterpret_cast<uint64_t *>(sm);            // window: outer key of element e
  uint64_t *const sorted = s_ko;                                      // placement: keys by digit
  uint32_t *const s_delta = reinterpret_cast<uint32_t *>(s_ko + kScRound);
  DigitDesc *const desc = reinterpret_cast<DigitDesc *>(s_delta + kScRound);
  uint32_t *const hist = reinterpret_cast<uint32_t *>(desc + nd);
  uint32_t *const loff = hist + nd;
  uint32_t *const bm = loff + nd;
  __shared__ uint32_t s_wt[32];
  __shared__ ScatterUnit u;
  __shared__ long long s_next_o;
  __shared__ uint32_t s_next_j;

  const int lanei = static_cast<int>(lane());
  const uint32_t lemask = (2u << lanei) - 1u;  // lanes <= this lane
  for (int i = threadIdx.x; i < nd; i += kScT) hist[i] = 0;

  for (int wu = blockIdx.x; wu < nwu; wu += gridDim.x) {
    __syncthreads();  // the previous unit's last round has read u
    if (threadIdx.x == 0) {
      const int per_inst = p.nclass * (p.slices[0] + p.slices[1]);
      const int inst_i = wu / per_inst;
      const FastInst &fi = p.inst[inst_i];
      const int nb0 = p.nclass * p.slices[0];
      int b = wu % per_inst;
      int side = 0;
      if (b >= nb0) {
        side = 1;
        b -= nb0;
      }
      const int ns = side ? p.slices[1] : p.slices[0];
      const int cl = b / ns, sl = b % ns;
      const SideGen &g = fi.side[side];
      const uint32_t cg_id = static_cast<uint32_t>(p.c0 + cl);
      u.okey = g.okey;
      u.ocls = g.ocls;
      u.ikey = g.ikey;
      u.ioff = g.ioff;
      u.isize = g.isize;
      u.rec = side ? p.rec[1] : p.rec[0];
      u.fill = fi.fill[side] + (int64_t)cl * nd;
      u.seg0 = fi.class_base[side][cg_id];
      u.o_cur = (int64_t)sl * g.slice_outer;
      u.o_end = min((int64_t)(sl + 1) * g.slice_outer, g.osize);
      u.j_cur = 0;
      u.cap = fi.cap[side][cg_id];
      u.r = cg_id & p.cmask;
      u.wmax = static_cast<uint32_t>(g.wmax);
      u.inst = inst_i;
    }
    __syncthreads();

    // the first slice of the next window, loaded during the current round
    bool pf_ok = false;  // block-uniform
    uint64_t pf_ko = 0;
    uint32_t pf_cls = 0, pf_ib = 0, pf_c = 0;
    while (u.o_cur < u.o_end) {
      // ---- 1. window: element idx = e * kScT + thread (coalesced) ----
      const long long o_cur = u.o_cur;
      const uint32_t j_cur = u.j_cur;
      const int w_n = static_cast<int>(min(static_cast<long long>(u.wmax), u.o_end - o_cur));
      uint32_t cnt[kScE], ibv[kScE];
      uint64_t kov[kScE];
      {
        const uint32_t *__restrict__ ocls = u.ocls;
        const uint32_t *__restrict__ ioff = u.ioff;
        const uint64_t *__restrict__ okey = u.okey;
        const uint32_t r = u.r, cmask = p.cmask;
#pragma unroll
        for (int e = 0; e < kScE; ++e) {
          const int idx = e * kScT + threadIdx.x;
          cnt[e] = 0;
          ibv[e] = 0;
          kov[e] = 0;
          // clamped so that the addresses stay inside the slice for every lane
          const long long o = o_cur + min(idx, w_n - 1);
          if (idx < w_n) {
            uint32_t ib, c;
            if (e == 0 && pf_ok) {
              kov[e] = pf_ko;
              ib = pf_ib;
              c = pf_c;
            } else {
              kov[e] = okey[o];
              const uint32_t w = (r - ocls[o]) & cmask;
              ib = ioff[w];
              c = ioff[w + 1] - ib;
            }
            if (idx == 0) {
              ib += j_cur;
              c -= j_cur;
            }
            cnt[e] = c;
            ibv[e] = ib;
          }
        }
      }
      for (int i = threadIdx.x; i < kScWords; i += kScT) bm[i] = 0;
      if (threadIdx.x == 0) {
        s_next_o = o_cur + w_n;
        s_next_j = 0;
      }
      // Element slices in order; a 32-bit scan per slice (records in the
      // high 22 bits, nonempty elements in the low 10) gives each element its
      // first record and its compacted position.  Counts enter the scan
      // clamped to kScRound + 1: every prefix that decides something (a
      // first record below kScRound, the element holding record kScRound,
      // the round's total when it is at most kScRound) is then exact.
      static_assert(kScT <= 1024 && kScT * (kScRound + 1) < (1u << 22), "packed window scan");
      unsigned long long rec_carry = 0;
      uint32_t pos_carry = 0;
#pragma unroll
      for (int e = 0; e < kScE; ++e) {
        if (e * kScT >= w_n) break;  // block-uniform
        const uint32_t c = cnt[e];
        const uint32_t cc = min(c, static_cast<uint32_t>(kScRound + 1));
        uint32_t tot_packed;
        // a further slice scans again; after the last one the block
        // barrier below comes first
        const uint32_t ex = scan_excl<uint32_t>((cc << 10) | (c ? 1u : 0u), s_wt, &tot_packed,
                                                (e + 1) * kScT < w_n);
        if (c) {
          const int idx = e * kScT + threadIdx.x;
          const unsigned long long pre = rec_carry + (ex >> 10);
          if (pre < kScRound) {
            const uint32_t pos = pos_carry + (ex & 0x3ffu);
            s_ko[pos] = kov[e];
            s_delta[pos] = ibv[e] - static_cast<uint32_t>(pre);
            atomicOr(&bm[pre >> 5], 1u << (pre & 31));
          }
          if (pre <= kScRound && pre + c > kScRound) {  // the element holding record kScRound
            s_next_o = o_cur + idx;
            s_next_j = static_cast<uint32_t>(kScRound - pre) + (idx == 0 ? j_cur : 0u);
          }
        }
        rec_carry += tot_packed >> 10;
        pos_carry += tot_packed & 0x3ffu;
      }
      const unsigned long long total = rec_carry;
      const uint32_t n_round = static_cast<uint32_t>(min(static_cast<unsigned long long>(kScRound), total));
      __syncthreads();
      {
        // the next window starts at s_next_o: load its first slice now
        const long long o_nx = s_next_o;
        const long long o_end = u.o_end;
        pf_ok = o_nx < o_end;
        if (pf_ok) {
          const int wn_nx = static_cast<int>(min(static_cast<long long>(u.wmax), o_end - o_nx));
          const long long o = o_nx + min(static_cast<int>(threadIdx.x), wn_nx - 1);
          pf_ko = u.okey[o];
          pf_cls = u.ocls[o];
        }
      }

      // ---- 2. generation: records [256 warp, 256 warp + 256) ----
      uint64_t keys[kScPer];
      uint32_t rank[kScPer];
      const uint32_t K0 = (threadIdx.x >> 5) * (kScPer * 32);
      if (K0 < n_round) {
        const uint64_t *__restrict__ ikey = u.ikey;
        // elements starting before K0: popcount of bitmap words [0, K0 / 32)
        const uint32_t w0 = K0 >> 5;
        uint32_t c0 = 0;
#pragma unroll
        for (int q = 0; q < (kScWords + 31) / 32; ++q) {
          const uint32_t wi = static_cast<uint32_t>(lanei + 32 * q);
          c0 += wi < w0 ? __popc(bm[wi]) : 0u;
        }
        uint32_t e_base = __reduce_add_sync(0xffffffffu, c0);
        // all gathers of the warp's records are issued before the first
        // shared atomic, so their latencies overlap
#pragma unroll
        for (int b = 0; b < kScPer; ++b) {
          const uint32_t K = K0 + b * 32;
          const uint32_t word = bm[K >> 5];
          uint32_t e = e_base + __popc(word & lemask) - 1u;
          e_base += __popc(word);
          const uint32_t k = K + lanei;
          if (k < n_round && !MSP_IN_BOUNDS(e, static_cast<uint32_t>(kScRound), 41u)) e = 0u;  // element
          rank[b] = e;  // element of the record until the rank replaces it
          // lanes past the round read inner element 0: every address formed
          // here is inside the inner list whether or not the load is
          // predicated
          uint32_t ii = k < n_round ? s_delta[e] + k : 0u;
          if (!MSP_IN_BOUNDS(ii, static_cast<uint64_t>(u.isize), 42u)) ii = 0u;  // inner position
          keys[b] = __ldg(ikey + ii);
        }
#pragma unroll
        for (int b = 0; b < kScPer; ++b) {
          const uint32_t k = K0 + b * 32 + lanei;
          if (k < n_round) {
            const uint64_t key = keys[b] + s_ko[rank[b]];
            keys[b] = key;
            rank[b] = atomicAdd(&hist[digit_t<D>(key)], 1u);
          }
        }
      }
      if (pf_ok) {  // bucket of the prefetched elements
        const uint32_t w = (u.r - pf_cls) & p.cmask;
        pf_ib = u.ioff[w];
        pf_c = u.ioff[w + 1] - pf_ib;
      }
      if (threadIdx.x == 0) {
        u.o_cur = s_next_o;  // read by the loop test after the barriers below
        u.j_cur = s_next_j;
      }
      __syncthreads();

      // ---- 3. digit offsets; one reservation per nonempty digit ----
      // The reservations are issued first; their results are needed only for
      // the run descriptors, which are formed after the placement, so the
      // atomics' latency hides behind the scan and the placement.
      uint32_t hv[pd], bv[pd], ov[pd];
      {
        uint32_t hsum = 0;
#pragma unroll
        for (int q = 0; q < pd; ++q) {
          const int gd = threadIdx.x * pd + q;
          hv[q] = gd < nd ? hist[min(gd, nd - 1)] : 0u;
          hsum += hv[q];
        }
        uint32_t *const fill = u.fill;
#pragma unroll
        for (int q = 0; q < pd; ++q) bv[q] = hv[q] ? atomicAdd(fill + threadIdx.x * pd + q, hv[q]) : 0u;
        uint32_t htot;
        uint32_t o = scan_excl<uint32_t>(hsum, s_wt, &htot, false);  // a block barrier follows
#pragma unroll
        for (int q = 0; q < pd; ++q) {
          const int gd = threadIdx.x * pd + q;
          ov[q] = o;
          if (gd < nd) {
            loff[gd] = o;
            hist[gd] = 0;
          }
          o += hv[q];
        }
      }
      __syncthreads();
      // ---- 4. place by digit, form the run descriptors, write the runs ----
      if (K0 < n_round) {
#pragma unroll
        for (int b = 0; b < kScPer; ++b) {
          const uint32_t k = K0 + b * 32 + lanei;
          if (k < n_round) {
            const uint32_t sp = loff[digit_t<D>(keys[b])] + rank[b];
            if (MSP_IN_BOUNDS(sp, static_cast<uint32_t>(kScRound), 43u)) sorted[sp] = keys[b];  // sorted slot
          }
        }
      }
      {
        const uint32_t cap = u.cap;
        const unsigned long long seg0 = u.seg0;
        bool ovf = false;
#pragma unroll
        for (int q = 0; q < pd; ++q) {
          const int gd = threadIdx.x * pd + q;
          const uint32_t h = hv[q];
          if (gd < nd && h) {
            const uint32_t base = bv[q];
            const uint32_t fit = base < cap ? min(h, cap - base) : 0u;
            ovf |= fit < h;
            DigitDesc dd;
            // may point before the partition; only positions from ov[q] on are used
            dd.dst = u.rec + (seg0 + (unsigned long long)gd * cap + base - ov[q]);
            dd.lim = ov[q] + fit;
            dd.pad = 0;
            desc[gd] = dd;
          }
        }
        if (ovf) atomicOr(p.overflow + u.inst, 1u);
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < kScPer; ++q) {
        const uint32_t i = threadIdx.x + q * kScT;
        if (i < n_round) {
          const uint64_t key = sorted[i];
          const DigitDesc dd = desc[digit_t<D>(key)];
          if (i < dd.lim) dd.dst[i] = key;
        }
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
// Join (S4 second digit + S5).  Persistent, two blocks of 512 threads per
// SM.  Partition s = (class, digit).  Thread 0 resolves the next
// partition's descriptor (where its keys lie, how many) and starts its left
// keys by cp.async.bulk into a shared buffer one partition ahead.  The left
// keys are hashed into a shared table of 2048 buckets (the 11 key bits below
// the digit) with 8 slots each; a slot holds a 16-bit fingerprint (the next
// key bits) and the key's 16-bit index in the partition, and a bucket past 8
// keys spills into a short overflow list.  Only the bucket counts are
// cleared between partitions: slots past a count are stale and never
// confirmed.  The right keys are read straight from device memory with
// coalesced 128-bit loads into registers (each is used once) and probe their
// bucket: one 128-bit shared load and four fingerprint compares for most
// buckets.  A fingerprint hit is confirmed against the full left key in
// device memory; the smallest index of an equal left key is claimed with a
// shared bit (so duplicate right keys emit once) and the (class, key) pair
// is appended with one atomic per warp.
// -------------------------------------------------------------------------
constexpr int kJT = 512;                    // threads per block, two blocks per SM
constexpr int kJBits = 11;                  // buckets of the probe table
constexpr int kJBuckets = 1 << kJBits;
constexpr int kJSlots = 8;                  // slots per bucket
constexpr int kJOvf = 512;                  // overflow entries (bucket << 16 | index)
constexpr int kJPairs = (kFastCap / 2 + kJT - 1) / kJT;  // 128-bit right loads per thread
static_assert(kFastCap <= 65536, "16-bit slot indices");
static_assert(kFastCap % 16 == 0, "partitions are 16-record multiples");

size_t join_fast_smem() {
  return (size_t)kFastCap * sizeof(uint64_t)                    // left keys (bulk copy target)
         + (size_t)kJBuckets * kJSlots * sizeof(uint16_t) * 2  // slot fingerprints, slot indices
         + (size_t)kJBuckets * sizeof(uint32_t)                // bucket fill
         + (size_t)(kFastCap / 32 + 1) * sizeof(uint32_t)      // claim bits
         + (size_t)kJOvf * sizeof(uint32_t)                    // overflow list
         + 64;
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

// Bounded wait on an mbarrier phase: thread 0 waits (limit_ns, 2 s by
// default; then it sets the error flag and waits once more, bounded by the
// same limit, so that a copy still in flight lands before the block exits),
// the block learns the outcome through shared memory, then every thread
// observes the completed phase.
__device__ __forceinline__ bool wait_phase(uint64_t *bar, uint32_t parity, unsigned int *err, int *s_ok,
                                           uint64_t limit_ns) {
  if (threadIdx.x == 0) {
    const uint64_t t0 = global_ns();
    bool ok = true;
    while (!mbar_try_wait(bar, parity)) {
      if (global_ns() - t0 > limit_ns) {
        ok = false;
        break;
      }
    }
    if (!ok) {
      atomicOr(err, 1u);
      const uint64_t t1 = global_ns();
      while (!mbar_try_wait(bar, parity) && global_ns() - t1 < limit_ns) {
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

// Bucket and fingerprint of a key: the kJBits bits below the top D (digit)
// bits, then 16 more (a key whose 16 bits are 0 uses 1, so that a slot of
// the zeroed table never matches).
template <int D>
__device__ __forceinline__ uint32_t jbucket(uint64_t key) {
  return static_cast<uint32_t>(key >> (64 - D - kJBits)) & (kJBuckets - 1u);
}
template <int D>
__device__ __forceinline__ uint32_t jfp(uint64_t key) {
  static_assert(D + kJBits + 16 <= 64, "fingerprint must fit below the digit");
  const uint32_t f = static_cast<uint32_t>(key >> (64 - D - kJBits - 16)) & 0xffffu;
  return f ? f : 1u;
}

// Nonzero when some 16-bit half of x is zero.
__device__ __forceinline__ uint32_t zero_half(uint32_t x) { return (x - 0x00010001u) & ~x & 0x80008000u; }

// Probe one right key.  Returns true when this lane claimed the lowest index
// of a left key equal to it.
template <int D>
__device__ __forceinline__ bool probe(uint64_t key, const uint64_t *__restrict__ Lg, const uint16_t *fps,
                                      const uint16_t *idxs, const uint32_t *cnt, const uint32_t *ovf,
                                      uint32_t n_ovf, uint32_t *flags) {
  const uint32_t b = jbucket<D>(key);
  const uint32_t fp = jfp<D>(key);
  // all 8 slots are compared at once; slots past the count hold stale
  // fingerprints of earlier partitions, so a hit is confirmed below on the
  // counted slots only
  const uint4 w = *reinterpret_cast<const uint4 *>(fps + b * kJSlots);
  const uint32_t f2 = fp * 0x00010001u;
  const uint32_t any = zero_half(w.x ^ f2) | zero_half(w.y ^ f2) | zero_half(w.z ^ f2) | zero_half(w.w ^ f2);
  const uint32_t c = cnt[b];
  if (!any && c <= kJSlots) return false;
  uint32_t best = 0xffffffffu;
  const uint32_t n = min(c, static_cast<uint32_t>(kJSlots));
  for (uint32_t j = 0; j < n; ++j) {
    if (fps[b * kJSlots + j] == fp) {
      const uint32_t idx = idxs[b * kJSlots + j];
      if (idx < best && MSP_IN_BOUNDS(idx, static_cast<uint32_t>(kFastCap), 44u) && Lg[idx] == key) best = idx;
    }
  }
  if (c > kJSlots) {
    for (uint32_t j = 0; j < n_ovf; ++j) {
      const uint32_t v = ovf[j];
      if ((v >> 16) == b) {
        const uint32_t idx = v & 0xffffu;
        if (idx < best && Lg[idx] == key) best = idx;
      }
    }
  }
  if (best == 0xffffffffu) return false;
  const uint32_t bit = 1u << (best & 31);
  return (atomicOr(&flags[best >> 5], bit) & bit) == 0;
}

template <int D>
__global__ void __launch_bounds__(kJT, 2) join_fast_kernel(FastPass p, int nseg) {
  extern __shared__ __align__(16) uint8_t sm[];
  uint64_t *const bufL = reinterpret_cast<uint64_t *>(sm);
  uint16_t *const fps = reinterpret_cast<uint16_t *>(bufL + kFastCap);
  uint16_t *const idxs = fps + kJBuckets * kJSlots;
  uint32_t *const cnt = reinterpret_cast<uint32_t *>(idxs + kJBuckets * kJSlots);
  uint32_t *const flags = cnt + kJBuckets;
  uint32_t *const ovf = flags + (kFastCap / 32 + 1);
  constexpr int nflag = kFastCap / 32 + 1;
  constexpr int nfp16 = kJBuckets * kJSlots / 8;  // fingerprint table in 16-byte words
  __shared__ __align__(8) uint64_t barL;
  __shared__ __align__(8) uint64_t barCheck;
  __shared__ uint32_t s_novf;
  __shared__ int s_ok;
  // the partition of this iteration and of the next: thread 0 resolves the
  // next one when it issues its left keys, so the dependent loads of
  // seg_ref leave the critical path of the iteration
  __shared__ SegRef s_ref[2];
  if (threadIdx.x == 0) {
    mbar_init(&barL, 1);
    mbar_init(&barCheck, 1);
    s_novf = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = threadIdx.x; i < kJBuckets; i += kJT) cnt[i] = 0;
  for (int i = threadIdx.x; i < nflag; i += kJT) flags[i] = 0;
  for (int i = threadIdx.x; i < nfp16; i += kJT) reinterpret_cast<uint4 *>(fps)[i] = make_uint4(0, 0, 0, 0);
  __syncthreads();
  if (p.wait_check) {
    // check of the bounded wait: a phase that expects 16 bytes no copy will
    // deliver, so the wait runs out, sets the error flag and the block
    // returns (no copy of this block is in flight yet)
    if (threadIdx.x == 0) mbar_arrive_expect_tx(&barCheck, 16u);
    if (!wait_phase(&barCheck, 0u, p.error, &s_ok, p.wait_ns)) return;
  }
  const int G = gridDim.x;
  int s = blockIdx.x;
  if (s < nseg && threadIdx.x == 0) {
    const SegRef r0 = seg_ref(p, s);
    s_ref[0] = r0;
    issue_keys(r0.L, r0.nL, bufL, &barL);
  }
  __syncthreads();
  uint32_t phL = 0;
  for (uint32_t it = 0; s < nseg; s += G, ++it) {
    const SegRef r = s_ref[it & 1u];
    // right keys of this partition: coalesced 128-bit loads into registers,
    // in flight while the left side is hashed
    ulonglong2 rk[kJPairs];
    const uint32_t npair = (r.nR + 1u) >> 1;
#pragma unroll
    for (int q = 0; q < kJPairs; ++q) {
      const uint32_t pi = threadIdx.x + q * kJT;
      // clamped: every address formed is inside the partition
      const uint32_t pc = npair ? min(pi, npair - 1u) : 0u;
      rk[q] = npair ? __ldg(reinterpret_cast<const ulonglong2 *>(r.R) + pc) : make_ulonglong2(0, 0);
    }
    if (!wait_phase(&barL, phL, p.error, &s_ok, p.wait_ns)) return;
    phL ^= 1u;
    // hash the left side
    for (uint32_t i = threadIdx.x; i < r.nL; i += kJT) {
      const uint64_t key = bufL[i];
      const uint32_t b = jbucket<D>(key);
      const uint32_t slot = atomicAdd(&cnt[b], 1u);
      if (slot < kJSlots) {
        fps[b * kJSlots + slot] = static_cast<uint16_t>(jfp<D>(key));
        idxs[b * kJSlots + slot] = static_cast<uint16_t>(i);
      } else {
        const uint32_t o = atomicAdd(&s_novf, 1u);
        if (o < kJOvf) ovf[o] = (b << 16) | i;
      }
    }
    __syncthreads();
    const int sn = s + G;
    if (sn < nseg && threadIdx.x == 0) {
      fence_proxy_async();
      const SegRef rn = seg_ref(p, sn);
      s_ref[(it + 1u) & 1u] = rn;  // read after the barrier that ends this iteration
      issue_keys(rn.L, rn.nL, bufL, &barL);
    }
    const uint32_t n_ovf = s_novf;
    if (n_ovf > kJOvf) {
      // more spilled keys than the list holds: the instance's pass is re-run
      // on the exact path
      if (threadIdx.x == 0) atomicOr(p.overflow + s / (p.nclass << p.D), 1u);
    } else {
#pragma unroll
      for (int q = 0; q < kJPairs; ++q) {
        const uint32_t pi = threadIdx.x + q * kJT;
        if (q * kJT < static_cast<int>(npair)) {  // block-uniform: bounds the emit calls
          const bool v0 = 2 * pi < r.nR, v1 = 2 * pi + 1 < r.nR;
          const bool e0 = v0 && probe<D>(rk[q].x, r.L, fps, idxs, cnt, ovf, n_ovf, flags);
          emit(p, e0, rk[q].x, r.cls);
          const bool e1 = v1 && probe<D>(rk[q].y, r.L, fps, idxs, cnt, ovf, n_ovf, flags);
          emit(p, e1, rk[q].y, r.cls);
        }
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kJBuckets; i += kJT) cnt[i] = 0;
    for (int i = threadIdx.x; i < nflag; i += kJT) flags[i] = 0;
    // the fingerprints are not cleared: slots past a bucket's count are
    // stale, and probe() confirms a fingerprint hit only on counted slots
    if (threadIdx.x == 0) s_novf = 0;
    // the next wait_phase begins with a block barrier
  }
}

template <int D>
static cudaError_t launch_join_d(const FastPass &p, int nclass_run, cudaStream_t s) {
  static size_t attr = 0;
  static int sms = 0, per_sm = 0;
  const size_t smem = join_fast_smem();
  if (smem > attr) {
    cudaError_t e = cudaFuncSetAttribute(join_fast_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    attr = smem;
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, join_fast_kernel<D>, kJT, smem) != cudaSuccess ||
        n < 1) {
      cudaGetLastError();
      n = 1;
    }
    per_sm = n;
  }
  FastPass q = p;
  q.nclass = nclass_run;
  const int nseg = p.ninst * (nclass_run << D);
  const int blocks = std::min(nseg, per_sm * sms);
  if (blocks < 1) return cudaSuccess;
  join_fast_kernel<D><<<blocks, kJT, smem, s>>>(q, nseg);
  return cudaGetLastError();
}

cudaError_t launch_join_fast(const FastPass &p, int nclass_run, cudaStream_t s) {
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
