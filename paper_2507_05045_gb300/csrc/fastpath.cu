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

__device__ __forceinline__ uint32_t digit_of(uint64_t key, int D) {
  return D ? static_cast<uint32_t>(key >> (64 - D)) : 0u;
}

__device__ __forceinline__ uint32_t subkey_of(uint64_t key, int D, int S) {
  return static_cast<uint32_t>((key >> (64 - D - S)) & ((1ull << S) - 1));
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

// Exclusive scan of a shared array of n entries in place (n <= 16 * blockDim).
__device__ void scan_array(uint32_t *a, int n, uint32_t *wt, uint32_t *total) {
  const int per = (n + blockDim.x - 1) / blockDim.x;
  uint32_t loc[16];
  uint32_t s = 0;
  for (int k = 0; k < per; ++k) {
    const int i = threadIdx.x * per + k;
    loc[k] = i < n ? a[i] : 0u;
    s += loc[k];
  }
  uint32_t ex = scan_excl<uint32_t>(s, wt, total);
  for (int k = 0; k < per; ++k) {
    const int i = threadIdx.x * per + k;
    if (i < n) a[i] = ex;
    ex += loc[k];
  }
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
                                                          unsigned long long *out) {
  __shared__ uint32_t sO[kCsU];
  __shared__ uint32_t sI[kCsU + kCsR];
  const uint32_t r0 = blockIdx.x * kCsR;
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
    if (r < M) {
      // u = u0 + i  ->  k = (r - r0) + (nu - 1) - i
      const uint32_t kb = threadIdx.x + (nu - 1);
      for (uint32_t i = 0; i < nu; ++i) acc += static_cast<unsigned long long>(sO[i]) * sI[kb - i];
    }
    __syncthreads();
  }
  if (r < M) out[r] = acc;
}

cudaError_t launch_class_sizes(const uint32_t *offO, const uint32_t *offI, uint32_t M, unsigned long long *out,
                               cudaStream_t s) {
  const uint32_t blocks = (M + kCsR - 1) / kCsR;
  class_size_kernel<<<blocks, kCsR, 0, s>>>(offO, offI, M, out);
  return cudaGetLastError();
}

// -------------------------------------------------------------------------
// Cluster scatter.
// -------------------------------------------------------------------------
constexpr int kCL = 8;          // blocks per cluster
constexpr int kScT = 256;       // threads per block
constexpr int kScPer = 32;      // records per thread per round
constexpr int kScChunk = kScT * kScPer;  // 8192 records per block per round
constexpr int kScE = 8;         // outer elements per thread in a window
constexpr int kScW = kScT * kScE;        // 2048 outer elements per window

size_t scatter_fast_smem(int D) {
  const size_t nd = size_t(1) << D;
  return kScChunk * sizeof(uint64_t)      // sorted records
         + kScW * sizeof(uint64_t)        // outer keys of the window
         + kScW * sizeof(uint32_t)        // inner bucket starts
         + (kScW + 1) * sizeof(uint32_t)  // record prefix of the window
         + 4 * nd * sizeof(uint32_t)      // hist, local offsets, cursors, cluster positions
         + 64;
}

__global__ void __cluster_dims__(kCL, 1, 1) __launch_bounds__(kScT, 2)
    scatter_fast_kernel(FastPass p, int nwu) {
  extern __shared__ __align__(16) uint8_t sm[];
  cg::cluster_group cluster = cg::this_cluster();
  const unsigned brank = cluster.block_rank();
  const int D = p.D;
  const int nd = 1 << D;
  uint64_t *sorted = reinterpret_cast<uint64_t *>(sm);
  uint64_t *s_ko = sorted + kScChunk;
  uint32_t *s_ib = reinterpret_cast<uint32_t *>(s_ko + kScW);
  uint32_t *s_pre = s_ib + kScW;
  uint32_t *hist = s_pre + kScW + 1;
  uint32_t *loff = hist + nd;
  uint32_t *cur = loff + nd;
  uint32_t *gpos = cur + nd;
  __shared__ uint32_t s_wt[32];
  __shared__ int s_active;

  const int ncl = gridDim.x / kCL;
  const int cid = blockIdx.x / kCL;
  for (int wu = cid; wu < nwu; wu += ncl) {
    // work unit -> (side, class, slice)
    int side, cl, sl;
    {
      const int nb0 = p.nclass * p.side[0].slices;
      int b = wu;
      if (b < nb0) {
        side = 0;
      } else {
        side = 1;
        b -= nb0;
      }
      cl = b / p.side[side].slices;
      sl = b % p.side[side].slices;
    }
    const SideGen &g = p.side[side];
    const uint32_t r = static_cast<uint32_t>(p.c0 + cl) & p.cmask;
    const int64_t s_begin = (int64_t)sl * g.slice_outer;
    const int64_t s_end = min(s_begin + g.slice_outer, g.osize);
    const int64_t part = (s_end - s_begin + kCL - 1) / kCL;
    const int64_t o_end = min(s_begin + part * (brank + 1), s_end);
    int64_t o_cur = min(s_begin + part * brank, s_end);
    uint32_t j_cur = 0;
    const uint32_t cap = p.cap[side][cl];
    uint64_t *const seg0 = p.rec[side] + p.class_base[side][cl];
    uint32_t *const fill = p.fill[side] + (int64_t)cl * nd;

    for (;;) {
      const bool active = o_cur < o_end;
      // ---- window of outer elements and the prefix of their records ----
      const int64_t w_n = active ? min(static_cast<int64_t>(kScW), o_end - o_cur) : 0;
      uint32_t cnt_loc[kScE];
      uint32_t tsum = 0;
#pragma unroll
      for (int e = 0; e < kScE; ++e) {
        const int idx = threadIdx.x * kScE + e;
        uint32_t c = 0;
        if (idx < w_n) {
          const int64_t o = o_cur + idx;
          const uint32_t w = (r - g.ocls[o]) & p.cmask;
          uint32_t ib = g.ioff[w];
          c = g.ioff[w + 1] - ib;
          if (idx == 0) {
            ib += j_cur;
            c -= j_cur;
          }
          s_ko[idx] = g.okey[o];
          s_ib[idx] = ib;
        }
        cnt_loc[e] = c;
        tsum += c;
      }
      for (int i = threadIdx.x; i < nd; i += kScT) hist[i] = 0;
      uint32_t total;
      uint32_t ex = scan_excl<uint32_t>(tsum, s_wt, &total);
#pragma unroll
      for (int e = 0; e < kScE; ++e) {
        s_pre[threadIdx.x * kScE + e] = ex;
        ex += cnt_loc[e];
      }
      if (threadIdx.x == 0) {
        s_pre[kScW] = total;
        s_active = active ? 1 : 0;
      }
      __syncthreads();
      const uint32_t n_round = min(static_cast<uint32_t>(kScChunk), total);

      // ---- generate this thread's records into registers ----
      uint64_t keys[kScPer];
      const uint32_t rb = threadIdx.x * kScPer;
      const uint32_t re = min(rb + kScPer, n_round);
      if (rb < re) {
        int lo = 0, hi = kScW - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (s_pre[mid] <= rb) lo = mid; else hi = mid - 1;
        }
        int e = lo;
        uint32_t j = rb - s_pre[e];
        uint32_t lim = s_pre[e + 1] - s_pre[e];
        uint64_t kob = s_ko[e];
        const uint64_t *ip = g.ikey + s_ib[e];
#pragma unroll
        for (int q = 0; q < kScPer; ++q) {
          if (rb + q < re) {
            while (j >= lim) {
              ++e;
              j = 0;
              lim = s_pre[e + 1] - s_pre[e];
              kob = s_ko[e];
              ip = g.ikey + s_ib[e];
            }
            keys[q] = kob + ip[j];
            ++j;
          }
        }
#pragma unroll
        for (int q = 0; q < kScPer; ++q)
          if (rb + q < re) atomicAdd(&hist[digit_of(keys[q], D)], 1u);
      }
      __syncthreads();
      // ---- advance the cursor past this round's records ----
      if (active) {
        if (n_round == total) {
          o_cur += w_n;
          j_cur = 0;
        } else {
          int lo = 0, hi = kScW - 1;
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_pre[mid] <= n_round) lo = mid; else hi = mid - 1;
          }
          j_cur = (n_round - s_pre[lo]) + (lo == 0 ? j_cur : 0u);
          o_cur += lo;
        }
      }
      // ---- local digit offsets ----
      for (int i = threadIdx.x; i < nd; i += kScT) loff[i] = hist[i];
      __syncthreads();
      uint32_t tot2;
      scan_array(loff, nd, s_wt, &tot2);
      for (int i = threadIdx.x; i < nd; i += kScT) cur[i] = loff[i];
      cluster.sync();  // #1: every block's histogram is final
      // ---- owners: cluster totals, one global reservation per digit ----
      int any = 0;
      for (unsigned b = 0; b < kCL; ++b) any |= *cluster.map_shared_rank(&s_active, b);
      for (int gd = brank + kCL * threadIdx.x; gd < nd; gd += kCL * kScT) {
        uint32_t h[kCL];
        uint32_t tot = 0;
#pragma unroll
        for (int b = 0; b < kCL; ++b) {
          h[b] = *cluster.map_shared_rank(hist + gd, b);
          tot += h[b];
        }
        if (tot) {
          uint32_t base = atomicAdd(fill + gd, tot);
#pragma unroll
          for (int b = 0; b < kCL; ++b) {
            *cluster.map_shared_rank(gpos + gd, b) = base;
            base += h[b];
          }
        }
      }
      cluster.sync();  // #2: positions delivered
      // ---- place by digit, then write the runs ----
      if (rb < re) {
#pragma unroll
        for (int q = 0; q < kScPer; ++q)
          if (rb + q < re) {
            const uint32_t pos = atomicAdd(&cur[digit_of(keys[q], D)], 1u);
            sorted[pos] = keys[q];
          }
      }
      __syncthreads();
      bool ovf = false;
      for (uint32_t i = threadIdx.x; i < n_round; i += kScT) {
        const uint64_t key = sorted[i];
        const uint32_t gd = digit_of(key, D);
        const uint32_t rel = gpos[gd] + (i - loff[gd]);
        if (rel < cap) seg0[(uint64_t)gd * cap + rel] = key; else ovf = true;
      }
      if (ovf) atomicOr(p.overflow, 1u);
      __syncthreads();
      if (!any) break;
    }
  }
}

cudaError_t launch_scatter_fast(const FastPass &p, int nclass_run, cudaStream_t s) {
  static size_t attr = 0;
  static int max_clusters = 0;
  const size_t smem = scatter_fast_smem(p.D);
  if (smem > attr) {
    cudaError_t e = cudaFuncSetAttribute(scatter_fast_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    attr = smem;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kCL * 64);
    cfg.blockDim = dim3(kScT);
    cfg.dynamicSmemBytes = smem;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, scatter_fast_kernel, &cfg) != cudaSuccess || n < 1) {
      cudaGetLastError();
      n = 16;
    }
    max_clusters = n;
  }
  FastPass q = p;
  q.nclass = nclass_run;
  const int nwu = nclass_run * (p.side[0].slices + p.side[1].slices);
  const int clusters = std::max(1, std::min(nwu, max_clusters));
  scatter_fast_kernel<<<clusters * kCL, kScT, smem, s>>>(q, nwu);
  return cudaGetLastError();
}

// -------------------------------------------------------------------------
// Persistent join with double-buffered bulk copies.
// -------------------------------------------------------------------------
constexpr int kJfT = 512;
constexpr int kJfReg = (kFastCap + kJfT - 1) / kJfT;

size_t join_fast_smem(int S) {
  return 4 * (size_t)kFastCap * sizeof(uint64_t) + 2 * (((size_t)1 << S) + 1) * sizeof(uint32_t) + 64;
}

struct SegRef {
  const uint64_t *L, *R;
  uint32_t nL, nR;
};

__device__ __forceinline__ SegRef seg_ref(const FastPass &p, int s) {
  const int nd = 1 << p.D;
  const int cl = s >> p.D, gd = s & (nd - 1);
  SegRef r;
  const uint32_t capL = p.cap[0][cl], capR = p.cap[1][cl];
  r.L = p.rec[0] + p.class_base[0][cl] + (uint64_t)gd * capL;
  r.R = p.rec[1] + p.class_base[1][cl] + (uint64_t)gd * capR;
  r.nL = min(p.fill[0][(int64_t)cl * nd + gd], capL);
  r.nR = min(p.fill[1][(int64_t)cl * nd + gd], capR);
  if (r.nL == 0 || r.nR == 0) r.nL = r.nR = 0;
  return r;
}

__device__ __forceinline__ void issue_seg(const SegRef &r, uint64_t *bufL, uint64_t *bufR, uint64_t *bar) {
  // sizes rounded up to 16 bytes; capacities are multiples of 16 records
  const uint32_t bl = ((r.nL + 1u) & ~1u) * 8u, br = ((r.nR + 1u) & ~1u) * 8u;
  mbar_arrive_expect_tx(bar, bl + br);
  if (bl) bulk_load(bufL, r.L, bl, bar);
  if (br) bulk_load(bufR, r.R, br, bar);
}

__device__ void sort_in_place(uint64_t *buf, uint32_t n, uint32_t *off, int D, int S, uint32_t *wt) {
  const int nb = 1 << S;
  uint64_t k[kJfReg];
  uint32_t rk[kJfReg];
#pragma unroll
  for (int q = 0; q < kJfReg; ++q) {
    const uint32_t i = threadIdx.x + q * kJfT;
    if (i < n) {
      k[q] = buf[i];
      rk[q] = atomicAdd(&off[subkey_of(k[q], D, S)], 1u);
    }
  }
  __syncthreads();
  uint32_t tot;
  scan_array(off, nb, wt, &tot);
  if (threadIdx.x == 0) off[nb] = tot;
#pragma unroll
  for (int q = 0; q < kJfReg; ++q) {
    const uint32_t i = threadIdx.x + q * kJfT;
    if (i < n) buf[off[subkey_of(k[q], D, S)] + rk[q]] = k[q];
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

__global__ void __launch_bounds__(kJfT, 1) join_fast_kernel(FastPass p, int nseg) {
  extern __shared__ __align__(16) uint8_t sm[];
  uint64_t *buf = reinterpret_cast<uint64_t *>(sm);  // [stage][side][kFastCap]
  const int S = p.S, D = p.D;
  const int nb = 1 << S;
  uint32_t *offL = reinterpret_cast<uint32_t *>(buf + 4 * kFastCap);
  uint32_t *offR = offL + nb + 1;
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t s_wt[32];
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int G = gridDim.x;
  int s = blockIdx.x;
  if (s < nseg && threadIdx.x == 0) issue_seg(seg_ref(p, s), buf, buf + kFastCap, &bar[0]);
  uint32_t phase[2] = {0, 0};
  for (int k = 0; s < nseg; ++k, s += G) {
    const int st = k & 1;
    uint64_t *bL = buf + (2 * st) * kFastCap;
    uint64_t *bR = bL + kFastCap;
    const int sn = s + G;
    if (sn < nseg && threadIdx.x == 0) {
      fence_proxy_async();
      uint64_t *nL = buf + (2 * (st ^ 1)) * kFastCap;
      issue_seg(seg_ref(p, sn), nL, nL + kFastCap, &bar[st ^ 1]);
    }
    const SegRef r = seg_ref(p, s);
    // bounded wait for this stage's copies: thread 0 decides for the block
    if (threadIdx.x == 0) {
      const uint64_t t0 = global_ns();
      bool ok = true;
      while (!mbar_try_wait(&bar[st], phase[st])) {
        if (global_ns() - t0 > 2000000000ull) {
          ok = false;
          break;
        }
      }
      if (!ok) {
        atomicOr(p.error, 1u);
        // give the copies in flight a last bounded chance to land
        const uint64_t t1 = global_ns();
        while (!mbar_try_wait(&bar[st], phase[st]) && global_ns() - t1 < 2000000000ull) {
        }
      }
      s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    if (!s_ok) return;
    // every thread observes the completed phase before reading the buffers
    while (!mbar_try_wait(&bar[st], phase[st])) {
    }
    phase[st] ^= 1u;
    if (r.nL && r.nR) {
      for (int i = threadIdx.x; i <= nb; i += kJfT) {
        offL[i] = 0;
        offR[i] = 0;
      }
      __syncthreads();
      sort_in_place(bL, r.nL, offL, D, S, s_wt);
      sort_in_place(bR, r.nR, offR, D, S, s_wt);
      __syncthreads();
      const uint32_t cls = static_cast<uint32_t>(p.c0 + (s >> D)) & p.cmask;
      const uint32_t rounds = (r.nL + kJfT - 1) / kJfT;
      for (uint32_t rd = 0; rd < rounds; ++rd) {
        const uint32_t i = rd * kJfT + threadIdx.x;
        bool e = false;
        uint64_t key = 0;
        if (i < r.nL) {
          key = bL[i];
          const uint32_t b = subkey_of(key, D, S);
          bool hit = false;
          for (uint32_t j = offR[b]; j < offR[b + 1]; ++j) hit |= (bR[j] == key);
          if (hit) {
            bool dup = false;
            for (uint32_t j = offL[b]; j < i; ++j) dup |= (bL[j] == key);
            e = !dup;
          }
        }
        emit(p, e, key, cls);
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_join_fast(const FastPass &p, int nclass_run, cudaStream_t s) {
  static size_t attr = 0;
  const size_t smem = join_fast_smem(p.S);
  if (smem > attr) {
    cudaError_t e = cudaFuncSetAttribute(join_fast_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    attr = smem;
  }
  const int nseg = nclass_run << p.D;
  int blocks = std::min(nseg, 152);
  if (blocks < 1) return cudaSuccess;
  join_fast_kernel<<<blocks, kJfT, smem, s>>>(p, nseg);
  return cudaGetLastError();
}

}  // namespace msp
