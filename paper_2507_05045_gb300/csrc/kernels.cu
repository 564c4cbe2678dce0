// Device kernels of libmsp (sm_103a).  Integer ALU and memory only: nothing
// on the path is a dense contraction, so no tensor-core code appears here.
//
// Steps (see msp_internal.cuh for the vocabulary):
//   gray_kernel            quarter subset-sum lists by Gray code (Algorithm 1,
//                          lists 2^A .. 2^D), all m row sums packed.
//   count_classes / bucket residue-class counting sort of the quarter lists
//                          (the partition of the row-1 key space).
//   gen_count/gen_scatter  per residue class, the half-pair records of L and
//                          R, radix-partitioned by the top key bits.
//   join_kernel            per partition: counting sort by the next key bits
//                          in shared memory and a bucket-aligned merge-join
//                          of L against R (Algorithm 3, sort + search).
//   recover / verify       the quarter elements behind each matched key and
//                          the exact all-row check A x = d (Algorithm 2).
#include "msp_internal.cuh"


namespace msp {

namespace {

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ uint32_t top_digit(uint64_t key, int D) {
  return D ? static_cast<uint32_t>(key >> (64 - D)) : 0u;
}

__device__ __forceinline__ uint32_t sub_key(uint64_t key, int D, int S) {
  return static_cast<uint32_t>((key >> (64 - D - S)) & ((1ull << S) - 1));
}

// Block-wide exclusive scan of one value per thread (blockDim.x <= 1024,
// a multiple of 32).  `warp_tot` needs 32 entries.  Returns the exclusive
// prefix; *total receives the block total.
template <typename T>
__device__ T block_exclusive_scan(T v, T *warp_tot, T *total) {
  const int lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T t = lane < nw ? warp_tot[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) warp_tot[lane] = t;  // inclusive per warp
  }
  __syncthreads();
  T before = warp ? warp_tot[warp - 1] : T(0);
  T incl = x + before;
  *total = warp_tot[nw - 1];
  __syncthreads();
  return incl - v;
}

}  // namespace

// -------------------------------------------------------------------------
// S1: quarter lists by Gray code.
// Thread c handles Gray ranks [c*chunk, (c+1)*chunk): it sums the columns of
// g(t0) directly, then walks the code; rank t flips column ctz(t), added if
// that bit of g(t) is set and removed otherwise.  Fields never leave
// [0, 2^16) because every partial row sum lies in [0, row sum].
// -------------------------------------------------------------------------
__global__ void gray_kernel(InstanceConst ic, const uint64_t *__restrict__ pcol,
                            const uint64_t *__restrict__ kcol, const uint32_t *__restrict__ ccol,
                            QuarterDev qd, int col0, int chunk) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t t0 = c * chunk;
  if (t0 >= qd.size) return;
  const int64_t t1 = min(t0 + (int64_t)chunk, qd.size);
  const int W = ic.W;
  const uint32_t cmask = (ic.class_bits >= 32) ? 0xffffffffu : ((1u << ic.class_bits) - 1u);
  uint64_t v[kMaxVecWords] = {0, 0, 0, 0};
  uint64_t k = 0;
  uint32_t cl = 0;
  const uint64_t g0 = static_cast<uint64_t>(t0 ^ (t0 >> 1));
  for (int j = 0; j < qd.q; ++j) {
    if ((g0 >> j) & 1) {
      const int col = col0 + j;
#pragma unroll
      for (int w = 0; w < kMaxVecWords; ++w)
        if (w < W) v[w] += pcol[col * kMaxVecWords + w];
      k += kcol[col];
      cl += ccol[col];
    }
  }
  for (int64_t t = t0;; ) {
#pragma unroll
    for (int w = 0; w < kMaxVecWords; ++w)
      if (w < W) qd.vec[w * qd.size + t] = v[w];
    qd.key[t] = k;
    qd.cls[t] = cl & cmask;
    qd.v1[t] = static_cast<uint32_t>(v[0] & 0xffffu);
    ++t;
    if (t >= t1) break;
    const int z = __ffsll(t) - 1;
    const int col = col0 + z;
    const bool in = ((static_cast<uint64_t>(t ^ (t >> 1)) >> z) & 1) != 0;
    if (in) {
#pragma unroll
      for (int w = 0; w < kMaxVecWords; ++w)
        if (w < W) v[w] += pcol[col * kMaxVecWords + w];
      k += kcol[col];
      cl += ccol[col];
    } else {
#pragma unroll
      for (int w = 0; w < kMaxVecWords; ++w)
        if (w < W) v[w] -= pcol[col * kMaxVecWords + w];
      k -= kcol[col];
      cl -= ccol[col];
    }
  }
}

cudaError_t launch_gray(const InstanceConst &ic, const uint64_t *pcol, const uint64_t *kcol,
                          const uint32_t *ccol, const QuarterDev &qd, int col0, cudaStream_t s) {
  int chunk = qd.size >= (1 << 16) ? 64 : 4;
  const int64_t threads = (qd.size + chunk - 1) / chunk;
  const int bs = 128;
  const int64_t blocks = (threads + bs - 1) / bs;
  gray_kernel<<<static_cast<unsigned>(blocks), bs, 0, s>>>(ic, pcol, kcol, ccol, qd, col0, chunk);
  return cudaGetLastError();
}

// -------------------------------------------------------------------------
// S2: residue classes.  Transformed class of an element: (mul*cls + add)&mask
// with mul = +1 for the left lists, -1 for Q2 (kappa(d) - kappa(c), add =
// kappa(d)) and Q4 (-kappa(e)).
// -------------------------------------------------------------------------
__global__ void count_classes_kernel(const uint32_t *__restrict__ cls, int64_t size, uint32_t mul,
                                     uint32_t add, uint32_t cmask, uint32_t *hist) {
  extern __shared__ uint32_t sh[];
  const bool use_smem = cmask < 4096u;
  if (use_smem) {
    for (uint32_t i = threadIdx.x; i <= cmask; i += blockDim.x) sh[i] = 0;
    __syncthreads();
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < size;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t c = (mul * cls[i] + add) & cmask;
    if (use_smem) atomicAdd(&sh[c], 1u); else atomicAdd(&hist[c], 1u);
  }
  if (use_smem) {
    __syncthreads();
    for (uint32_t i = threadIdx.x; i <= cmask; i += blockDim.x)
      if (sh[i]) atomicAdd(&hist[i], sh[i]);
  }
}

cudaError_t launch_count_classes(const uint32_t *cls, int64_t size, uint32_t mul, uint32_t add,
                                 uint32_t cmask, uint32_t *hist, cudaStream_t s) {
  const int bs = 256;
  int64_t blocks = (size + bs * 8 - 1) / (bs * 8);
  if (blocks < 1) blocks = 1;
  if (blocks > 4096) blocks = 4096;
  const size_t smem = cmask < 4096u ? (cmask + 1) * sizeof(uint32_t) : 0;
  count_classes_kernel<<<static_cast<unsigned>(blocks), bs, smem, s>>>(cls, size, mul, add, cmask, hist);
  return cudaGetLastError();
}

// Counting-sort scatter into class buckets.  Lanes of a warp with the same
// class are grouped by __match_any_sync so one atomic serves them all.
__global__ void bucket_scatter_kernel(QuarterDev qd, int64_t mul, uint64_t kadd, uint32_t cadd,
                                      uint32_t cmask, uint32_t *cursor, BucketDev bd) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t base0 = blockIdx.x * (int64_t)blockDim.x;
  for (int64_t b = base0; b < qd.size; b += stride) {
    const int64_t i = b + threadIdx.x;
    const bool ok = i < qd.size;
    uint32_t c = 0xffffffffu;
    uint64_t k = 0;
    if (ok) {
      c = (static_cast<uint32_t>(mul) * qd.cls[i] + cadd) & cmask;
      k = static_cast<uint64_t>(mul) * qd.key[i] + kadd;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (ok && static_cast<int>(lane_id()) == leader) base = atomicAdd(&cursor[c], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    if (ok) {
      const uint32_t pos = base + __popc(peers & ((1u << lane_id()) - 1u));
      bd.key[pos] = k;
      bd.cls[pos] = c;
      bd.idx[pos] = static_cast<uint32_t>(i);
    }
  }
}

cudaError_t launch_bucket_scatter(const QuarterDev &qd, int64_t mul, uint64_t kadd, uint32_t cadd,
                                  uint32_t cmask, uint32_t *cursor, const BucketDev &bd, cudaStream_t s) {
  const int bs = 256;
  int64_t blocks = (qd.size + bs - 1) / bs;
  if (blocks > 8192) blocks = 8192;
  bucket_scatter_kernel<<<static_cast<unsigned>(blocks), bs, 0, s>>>(qd, mul, kadd, cadd, cmask, cursor, bd);
  return cudaGetLastError();
}

// -------------------------------------------------------------------------
// Exclusive scans: out[i] = in[0] + ... + in[i-1] for i <= n (out has n+1
// entries, out[n] = total).  Three phases over tiles of 1024*4 elements.
// -------------------------------------------------------------------------
template <typename T>
__global__ void scan_tile_sums(const T *__restrict__ in, int64_t n, T *tile_sum) {
  __shared__ T wt[32];
  __shared__ T tot;
  const int64_t base = blockIdx.x * (int64_t)blockDim.x * 4;
  T s = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t i = base + threadIdx.x * 4 + k;
    if (i < n) s += in[i];
  }
  T t;
  block_exclusive_scan<T>(s, wt, &t);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = t;
  (void)tot;
}

template <typename T>
__global__ void scan_tile_sums_single(T *tile_sum, int64_t ntiles) {
  // one block: exclusive scan of tile sums in place, chunks of blockDim
  __shared__ T wt[32];
  T carry = 0;
  for (int64_t b = 0; b < ntiles; b += blockDim.x) {
    const int64_t i = b + threadIdx.x;
    const T v = i < ntiles ? tile_sum[i] : T(0);
    T tot;
    const T ex = block_exclusive_scan<T>(v, wt, &tot);
    if (i < ntiles) tile_sum[i] = ex + carry;
    carry += tot;
    __syncthreads();
  }
}

template <typename T>
__global__ void scan_apply(const T *__restrict__ in, T *out, int64_t n, const T *tile_sum) {
  __shared__ T wt[32];
  const int64_t base = blockIdx.x * (int64_t)blockDim.x * 4;
  T vals[4];
  T s = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t i = base + threadIdx.x * 4 + k;
    vals[k] = i < n ? in[i] : T(0);
    s += vals[k];
  }
  T tot;
  T ex = block_exclusive_scan<T>(s, wt, &tot) + tile_sum[blockIdx.x];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t i = base + threadIdx.x * 4 + k;
    if (i <= n) out[i] = ex;
    ex += vals[k];
  }
}

template <typename T>
static cudaError_t scan_impl(const T *in, T *out, int64_t n, T *tmp, cudaStream_t s) {
  // tmp must hold ceil((n+1)/4096) entries.  `in` and `out` may alias only
  // when in == out is not required; callers pass distinct buffers.
  const int bs = 1024;
  const int64_t per = bs * 4;
  const int64_t ntiles = (n + 1 + per - 1) / per;
  scan_tile_sums<T><<<static_cast<unsigned>(ntiles), bs, 0, s>>>(in, n, tmp);
  scan_tile_sums_single<T><<<1, bs, 0, s>>>(tmp, ntiles);
  scan_apply<T><<<static_cast<unsigned>(ntiles), bs, 0, s>>>(in, out, n, tmp);
  return cudaGetLastError();
}

cudaError_t launch_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *tmp, cudaStream_t s) {
  return scan_impl<uint32_t>(in, out, n, tmp, s);
}
cudaError_t launch_scan_u64(const unsigned long long *in, unsigned long long *out, int64_t n,
                            unsigned long long *tmp, cudaStream_t s) {
  return scan_impl<unsigned long long>(in, out, n, tmp, s);
}

// -------------------------------------------------------------------------
// Row-1 candidate count C1 = #{(l, r) : row1(l) + row1(r) = d_1}: histograms
// of the row-1 sums of each quarter, convolved per half, then the dot
// product sum_v hL[v] * hR[d_1 - v] in 128-bit arithmetic.
// -------------------------------------------------------------------------
__global__ void v1_hist_kernel(const uint32_t *__restrict__ v1, int64_t size, unsigned long long *hist) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < size;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&hist[v1[i]], 1ull);
}

cudaError_t launch_v1_hist(const uint32_t *v1, int64_t size, unsigned long long *hist, cudaStream_t s) {
  int64_t blocks = (size + 255) / 256;
  if (blocks > 2048) blocks = 2048;
  v1_hist_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(v1, size, hist);
  return cudaGetLastError();
}

__global__ void conv_kernel(const unsigned long long *a, int la, const unsigned long long *b, int lb,
                            unsigned long long *out, int lo) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= lo) return;
  unsigned long long s = 0;
  const int u0 = v - (lb - 1) > 0 ? v - (lb - 1) : 0;
  const int u1 = v < la - 1 ? v : la - 1;
  for (int u = u0; u <= u1; ++u) s += a[u] * b[v - u];
  out[v] = s;
}

__global__ void c1_dot_kernel(const unsigned long long *hl, int lenl, const unsigned long long *hr,
                              int lenr, int64_t d1, unsigned long long *out2) {
  __shared__ unsigned long long lo_s[1024], hi_s[1024];
  unsigned __int128 acc = 0;
  for (int64_t v = threadIdx.x; v < lenl; v += blockDim.x) {
    const int64_t w = d1 - v;
    if (w >= 0 && w < lenr) acc += static_cast<unsigned __int128>(hl[v]) * hr[w];
  }
  lo_s[threadIdx.x] = static_cast<unsigned long long>(acc);
  hi_s[threadIdx.x] = static_cast<unsigned long long>(acc >> 64);
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned __int128 t = 0;
    for (int i = 0; i < blockDim.x; ++i)
      t += (static_cast<unsigned __int128>(hi_s[i]) << 64) | lo_s[i];
    out2[0] = static_cast<unsigned long long>(t);
    out2[1] = static_cast<unsigned long long>(t >> 64);
  }
}

cudaError_t launch_row1_candidates(const unsigned long long *h1, const unsigned long long *h3, int len13,
                                   const unsigned long long *h2, const unsigned long long *h4, int len24,
                                   unsigned long long *hl, unsigned long long *hr, int lenl, int lenr,
                                   int64_t d1, unsigned long long *out2, cudaStream_t s) {
  conv_kernel<<<(lenl + 255) / 256, 256, 0, s>>>(h1, len13, h3, len13, hl, lenl);
  conv_kernel<<<(lenr + 255) / 256, 256, 0, s>>>(h2, len24, h4, len24, hr, lenr);
  c1_dot_kernel<<<1, 1024, 0, s>>>(hl, lenl, hr, lenr, d1, out2);
  return cudaGetLastError();
}

// -------------------------------------------------------------------------
// S3: half-pair records of one residue class.
// A block owns a slice (class r, outer range).  The outer range is walked in
// tiles of blockDim elements; each outer element o pairs with the inner
// bucket r - kappa(o).  A block scan of the bucket sizes flattens the tile's
// records, and every thread then takes a contiguous run of them.
// -------------------------------------------------------------------------
struct SliceRef {
  int side, cl, sl;
};

__device__ __forceinline__ SliceRef decode_slice(const PassDev &p, int64_t b) {
  SliceRef r;
  const int64_t nb0 = (int64_t)p.nclass * p.side[0].slices;
  if (b < nb0) {
    r.side = 0;
  } else {
    r.side = 1;
    b -= nb0;
  }
  const int sl = p.side[r.side].slices;
  r.cl = static_cast<int>(b / sl);
  r.sl = static_cast<int>(b % sl);
  return r;
}

// Visits every record of the slice: f(key) on the calling thread.
template <typename F>
__device__ __forceinline__ void for_each_record(const PassDev &p, const SliceRef &sr, F &&f) {
  __shared__ unsigned long long s_pre[kGenThreads + 1];
  __shared__ uint64_t s_ko[kGenThreads];
  __shared__ uint32_t s_ib[kGenThreads];
  __shared__ unsigned long long s_wt[32];
  const SideGen &g = p.side[sr.side];
  const uint32_t r = static_cast<uint32_t>(p.c0 + sr.cl) & p.cmask;
  const int64_t o_begin = (int64_t)sr.sl * g.slice_outer;
  const int64_t o_end = min(o_begin + g.slice_outer, g.osize);
  const int T = blockDim.x;
  for (int64_t base = o_begin; base < o_end; base += T) {
    const int64_t o = base + threadIdx.x;
    unsigned long long cnt = 0;
    uint64_t ko = 0;
    uint32_t ib = 0;
    if (o < o_end) {
      ko = g.okey[o];
      const uint32_t w = (r - g.ocls[o]) & p.cmask;
      ib = g.ioff[w];
      cnt = g.ioff[w + 1] - ib;
    }
    unsigned long long total;
    const unsigned long long pre = block_exclusive_scan<unsigned long long>(cnt, s_wt, &total);
    s_pre[threadIdx.x] = pre;
    s_ko[threadIdx.x] = ko;
    s_ib[threadIdx.x] = ib;
    if (threadIdx.x == 0) s_pre[T] = total;
    __syncthreads();
    const unsigned long long per = (total + T - 1) / T;
    unsigned long long k = per * threadIdx.x;
    const unsigned long long kend = min(k + per, total);
    if (k < kend) {
      // last outer element whose prefix is <= k
      int lo = 0, hi = T - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_pre[mid] <= k) lo = mid; else hi = mid - 1;
      }
      int ol = lo;
      unsigned long long j = k - s_pre[ol];
      uint64_t kob = s_ko[ol];
      const uint64_t *ip = g.ikey + s_ib[ol];
      unsigned long long lim = s_pre[ol + 1] - s_pre[ol];
      for (; k < kend; ++k) {
        while (j >= lim) {
          ++ol;
          j = 0;
          kob = s_ko[ol];
          ip = g.ikey + s_ib[ol];
          lim = s_pre[ol + 1] - s_pre[ol];
        }
        f(kob + ip[j]);
        ++j;
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kGenThreads) gen_count_kernel(PassDev p) {
  extern __shared__ uint32_t hist[];
  const SliceRef sr = decode_slice(p, blockIdx.x);
  const int nd = 1 << p.D;
  for (int i = threadIdx.x; i < nd; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  const int D = p.D;
  for_each_record(p, sr, [&](uint64_t key) { atomicAdd(&hist[top_digit(key, D)], 1u); });
  __syncthreads();
  uint32_t *dst = p.cnt[sr.side] + ((int64_t)sr.cl * p.side[sr.side].slices + sr.sl) * nd;
  for (int i = threadIdx.x; i < nd; i += blockDim.x) dst[i] = hist[i];
}

cudaError_t launch_gen_count(const PassDev &p, cudaStream_t s) {
  const int64_t blocks = (int64_t)p.nclass * (p.side[0].slices + p.side[1].slices);
  const size_t smem = sizeof(uint32_t) << p.D;
  gen_count_kernel<<<static_cast<unsigned>(blocks), kGenThreads, smem, s>>>(p);
  return cudaGetLastError();
}

// Per (side, class): turn the slice histograms into in-segment offsets, the
// segment lengths and starts, and the class total.
__global__ void counts_to_offsets_kernel(PassDev p) {
  __shared__ unsigned long long s_wt[32];
  const int side = blockIdx.x < static_cast<unsigned>(p.nclass) ? 0 : 1;
  const int cl = side ? blockIdx.x - p.nclass : blockIdx.x;
  const int nd = 1 << p.D;
  const int slices = p.side[side].slices;
  uint32_t *cnt = p.cnt[side] + (int64_t)cl * slices * nd;
  uint32_t *seglen = p.seglen[side] + (int64_t)cl * nd;
  uint64_t *segstart = p.segstart[side] + (int64_t)cl * nd;
  unsigned long long carry = 0;
  for (int g0 = 0; g0 < nd; g0 += blockDim.x) {
    const int g = g0 + threadIdx.x;
    unsigned long long len = 0;
    if (g < nd) {
      uint32_t run = 0;
      for (int sl = 0; sl < slices; ++sl) {
        const uint32_t c = cnt[(int64_t)sl * nd + g];
        cnt[(int64_t)sl * nd + g] = run;
        run += c;
      }
      seglen[g] = run;
      len = run;
    }
    unsigned long long tot;
    const unsigned long long ex = block_exclusive_scan<unsigned long long>(len, s_wt, &tot);
    if (g < nd) segstart[g] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) p.classtot[side][cl] = carry;
}

cudaError_t launch_counts_to_offsets(const PassDev &p, cudaStream_t s) {
  counts_to_offsets_kernel<<<2 * p.nclass, 256, 0, s>>>(p);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kGenThreads) gen_scatter_kernel(PassDev p, int nclass_run) {
  extern __shared__ uint32_t cursor[];
  SliceRef sr;
  {
    // blocks cover only the classes that fit: remap the block index
    int64_t b = blockIdx.x;
    const int64_t nb0 = (int64_t)nclass_run * p.side[0].slices;
    if (b < nb0) {
      sr.side = 0;
    } else {
      sr.side = 1;
      b -= nb0;
    }
    sr.cl = static_cast<int>(b / p.side[sr.side].slices);
    sr.sl = static_cast<int>(b % p.side[sr.side].slices);
  }
  const int nd = 1 << p.D;
  const uint32_t *off = p.cnt[sr.side] + ((int64_t)sr.cl * p.side[sr.side].slices + sr.sl) * nd;
  for (int i = threadIdx.x; i < nd; i += blockDim.x) cursor[i] = off[i];
  __syncthreads();
  const int D = p.D;
  uint64_t *out = p.rec[sr.side] + p.classbase[sr.side][sr.cl];
  const uint64_t *segstart = p.segstart[sr.side] + (int64_t)sr.cl * nd;
  for_each_record(p, sr, [&](uint64_t key) {
    const uint32_t dg = top_digit(key, D);
    const uint32_t pos = atomicAdd(&cursor[dg], 1u);
    out[segstart[dg] + pos] = key;
  });
}

cudaError_t launch_gen_scatter(const PassDev &p, int nclass_run, cudaStream_t s) {
  const int64_t blocks = (int64_t)nclass_run * (p.side[0].slices + p.side[1].slices);
  const size_t smem = sizeof(uint32_t) << p.D;
  gen_scatter_kernel<<<static_cast<unsigned>(blocks), kGenThreads, smem, s>>>(p, nclass_run);
  return cudaGetLastError();
}

// -------------------------------------------------------------------------
// S4 + S5: per partition (class, digit), counting sort of both sides by the
// S key bits below the digit in shared memory, then a bucket-aligned
// merge-join.  A left key is emitted once (first of its equal-key run in the
// bucket) when the right side holds the same key.
// -------------------------------------------------------------------------
struct JoinSmem {
  uint64_t *sL, *sR;
  uint32_t *offL, *offR;
};

__device__ __forceinline__ JoinSmem join_smem(uint8_t *smem, int S) {
  JoinSmem j;
  j.sL = reinterpret_cast<uint64_t *>(smem);
  j.sR = j.sL + kJoinCap;
  j.offL = reinterpret_cast<uint32_t *>(j.sR + kJoinCap);
  j.offR = j.offL + (1 << S) + 1;
  return j;
}

constexpr int kPerThread = kJoinCap / kJoinThreads;  // 12

// Load n <= kJoinCap keys from global, counting-sort them by sub_key into s;
// off[b] .. off[b+1] is bucket b afterwards.
__device__ void load_and_sort(const uint64_t *__restrict__ g, uint32_t n, uint64_t *s, uint32_t *off,
                              int D, int S) {
  __shared__ uint32_t s_wt[32];
  const int nb = 1 << S;
  for (int i = threadIdx.x; i <= nb; i += blockDim.x) off[i] = 0;
  __syncthreads();
  uint64_t keys[kPerThread];
  uint32_t rank[kPerThread];
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    const uint32_t i = threadIdx.x + k * blockDim.x;
    if (i < n) {
      keys[k] = g[i];
      rank[k] = atomicAdd(&off[sub_key(keys[k], D, S)], 1u);
    }
  }
  __syncthreads();
  // exclusive scan of the bucket counts (nb entries, nb / blockDim per thread)
  const int per = (nb + blockDim.x - 1) / blockDim.x;
  uint32_t local[8];
  uint32_t sum = 0;
  for (int k = 0; k < per; ++k) {
    const int i = threadIdx.x * per + k;
    local[k] = i < nb ? off[i] : 0;
    sum += local[k];
  }
  uint32_t tot;
  uint32_t ex = block_exclusive_scan<uint32_t>(sum, s_wt, &tot);
  for (int k = 0; k < per; ++k) {
    const int i = threadIdx.x * per + k;
    if (i < nb) off[i] = ex;
    ex += local[k];
  }
  if (threadIdx.x == 0) off[nb] = tot;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    const uint32_t i = threadIdx.x + k * blockDim.x;
    if (i < n) s[off[sub_key(keys[k], D, S)] + rank[k]] = keys[k];
  }
  __syncthreads();
}

__device__ __forceinline__ void emit_matches(const PassDev &p, bool emit, uint64_t key, uint32_t cls) {
  const unsigned bal = __ballot_sync(0xffffffffu, emit);
  if (!bal) return;
  const int leader = __ffs(bal) - 1;
  unsigned long long base = 0;
  if (static_cast<int>(lane_id()) == leader) base = atomicAdd(p.match_count, (unsigned long long)__popc(bal));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (emit) {
    const unsigned long long slot = base + __popc(bal & ((1u << lane_id()) - 1u));
    if (slot < p.match_cap) {
      p.match_key[slot] = key;
      p.match_cls[slot] = cls;
    }
  }
}

__global__ void __launch_bounds__(kJoinThreads) join_kernel(PassDev p) {
  extern __shared__ uint8_t smem[];
  const int D = p.D, S = p.S;
  const int nd = 1 << D;
  const int cl = blockIdx.x >> D;
  const int dg = blockIdx.x & (nd - 1);
  const uint32_t nL = p.seglen[0][(int64_t)cl * nd + dg];
  const uint32_t nR = p.seglen[1][(int64_t)cl * nd + dg];
  if (nL == 0 || nR == 0) return;
  if (nL > kJoinCap || nR > kJoinCap) {
    if (threadIdx.x == 0) {
      const unsigned slot = atomicAdd(p.big_count, 1u);
      if (slot < p.big_cap) p.big_list[slot] = (static_cast<uint32_t>(cl) << 16) | static_cast<uint32_t>(dg);
    }
    return;
  }
  const JoinSmem js = join_smem(smem, S);
  const uint64_t *gL = p.rec[0] + p.classbase[0][cl] + p.segstart[0][(int64_t)cl * nd + dg];
  const uint64_t *gR = p.rec[1] + p.classbase[1][cl] + p.segstart[1][(int64_t)cl * nd + dg];
  load_and_sort(gL, nL, js.sL, js.offL, D, S);
  load_and_sort(gR, nR, js.sR, js.offR, D, S);
  const uint32_t cls = static_cast<uint32_t>(p.c0 + cl) & p.cmask;
  const uint32_t rounds = (nL + blockDim.x - 1) / blockDim.x;
  for (uint32_t rd = 0; rd < rounds; ++rd) {
    const uint32_t i = rd * blockDim.x + threadIdx.x;
    bool emit = false;
    uint64_t key = 0;
    if (i < nL) {
      key = js.sL[i];
      const uint32_t b = sub_key(key, D, S);
      bool hit = false;
      for (uint32_t j = js.offR[b]; j < js.offR[b + 1]; ++j) hit |= (js.sR[j] == key);
      if (hit) {
        bool dup = false;
        for (uint32_t j = js.offL[b]; j < i; ++j) dup |= (js.sL[j] == key);
        emit = !dup;
      }
    }
    emit_matches(p, emit, key, cls);
  }
}

cudaError_t launch_join(const PassDev &p, int nclass_run, cudaStream_t s) {
  const size_t smem = 2 * kJoinCap * sizeof(uint64_t) + 2 * (((size_t)1 << p.S) + 1) * sizeof(uint32_t);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(join_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024);
    attr_set = true;
  }
  const int64_t blocks = (int64_t)nclass_run << p.D;
  join_kernel<<<static_cast<unsigned>(blocks), kJoinThreads, smem, s>>>(p);
  return cudaGetLastError();
}

// Oversize partitions: the left side in chunks of kJoinCap sorted in shared
// memory, the whole right side streamed against each chunk.  A key present
// in several left chunks is emitted once per chunk; the solution list is
// de-duplicated at the end.
__global__ void __launch_bounds__(kJoinThreads) join_big_kernel(PassDev p) {
  extern __shared__ uint8_t smem[];
  const int D = p.D, S = p.S;
  const int nd = 1 << D;
  const JoinSmem js = join_smem(smem, S);
  uint32_t *flag = reinterpret_cast<uint32_t *>(js.sR);  // reuse: kJoinCap flags
  const unsigned nbig = min(*p.big_count, p.big_cap);
  for (unsigned e = blockIdx.x; e < nbig; e += gridDim.x) {
    const uint32_t ent = p.big_list[e];
    const int cl = static_cast<int>(ent >> 16), dg = static_cast<int>(ent & 0xffffu);
    const uint32_t nL = p.seglen[0][(int64_t)cl * nd + dg];
    const uint32_t nR = p.seglen[1][(int64_t)cl * nd + dg];
    const uint64_t *gL = p.rec[0] + p.classbase[0][cl] + p.segstart[0][(int64_t)cl * nd + dg];
    const uint64_t *gR = p.rec[1] + p.classbase[1][cl] + p.segstart[1][(int64_t)cl * nd + dg];
    const uint32_t cls = static_cast<uint32_t>(p.c0 + cl) & p.cmask;
    for (uint32_t c0 = 0; c0 < nL; c0 += kJoinCap) {
      const uint32_t n = min(static_cast<uint32_t>(kJoinCap), nL - c0);
      load_and_sort(gL + c0, n, js.sL, js.offL, D, S);
      for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) flag[i] = 0;
      __syncthreads();
      for (uint32_t j = threadIdx.x; j < nR; j += blockDim.x) {
        const uint64_t key = gR[j];
        const uint32_t b = sub_key(key, D, S);
        for (uint32_t i = js.offL[b]; i < js.offL[b + 1]; ++i)
          if (js.sL[i] == key) flag[i] = 1;
      }
      __syncthreads();
      const uint32_t rounds = (n + blockDim.x - 1) / blockDim.x;
      for (uint32_t rd = 0; rd < rounds; ++rd) {
        const uint32_t i = rd * blockDim.x + threadIdx.x;
        bool emit = false;
        uint64_t key = 0;
        if (i < n && flag[i]) {
          key = js.sL[i];
          const uint32_t b = sub_key(key, D, S);
          bool dup = false;
          for (uint32_t j = js.offL[b]; j < i; ++j) dup |= (js.sL[j] == key);
          emit = !dup;
        }
        emit_matches(p, emit, key, cls);
      }
      __syncthreads();
    }
  }
}

cudaError_t launch_join_big(const PassDev &p, int nclass_run, cudaStream_t s) {
  (void)nclass_run;
  const size_t smem = 2 * kJoinCap * sizeof(uint64_t) + 2 * (((size_t)1 << p.S) + 1) * sizeof(uint32_t);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(join_big_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024);
    attr_set = true;
  }
  join_big_kernel<<<152, kJoinThreads, smem, s>>>(p);
  return cudaGetLastError();
}

// -------------------------------------------------------------------------
// S6: recovery and exact verification.
// For a matched (class r, key k) the left candidates are the pairs (a, b)
// with kappa(a) + kappa(b) = r and K(a) + K(b) = k: for every outer a the
// inner bucket r - kappa(a) is searched for k - K(a).  Same on the right.
// -------------------------------------------------------------------------
__global__ void recover_kernel(RecoverDev r, int side, bool emit) {
  const SideGen g = r.side[side];
  const uint64_t total = r.nmatch * static_cast<uint64_t>(g.osize);
  for (uint64_t idx = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t mi = idx / static_cast<uint64_t>(g.osize);
    const int64_t o = static_cast<int64_t>(idx - mi * static_cast<uint64_t>(g.osize));
    const uint64_t want = r.match_key[mi] - g.okey[o];
    const uint32_t w = (r.match_cls[mi] - g.ocls[o]) & r.cmask;
    const uint32_t jb = g.ioff[w], je = g.ioff[w + 1];
    for (uint32_t j = jb; j < je; ++j) {
      if (g.ikey[j] != want) continue;
      if (!emit) {
        atomicAdd(&r.cand_count[side][mi], 1ull);
      } else {
        const unsigned long long pos = r.cand_off[side][mi] + atomicAdd(&r.cand_cur[side][mi], 1ull);
        if (pos < r.cand_cap[side]) {
          r.cand[side][pos] = (static_cast<uint64_t>(r.oidx[side][o]) << 32) | r.iidx[side][j];
          if (side == 0) r.cand_match[0][pos] = static_cast<uint32_t>(mi);
        }
      }
    }
  }
}

cudaError_t launch_recover(const RecoverDev &r, bool emit, cudaStream_t s) {
  for (int side = 0; side < 2; ++side) {
    const uint64_t total = r.nmatch * static_cast<uint64_t>(r.side[side].osize);
    if (total == 0) continue;
    uint64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    recover_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(r, side, emit);
  }
  return cudaGetLastError();
}

__device__ __forceinline__ void add_mask(uint64_t m[2], uint64_t gray_rank, int col0) {
  const uint64_t g = gray_rank ^ (gray_rank >> 1);
  if (col0 < 64) {
    m[0] |= g << col0;
    if (col0 > 0) m[1] |= g >> (64 - col0);
  } else {
    m[1] |= g << (col0 - 64);
  }
}

__global__ void verify_kernel(VerifyDev v) {
  const int W = v.ic.W;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < v.nL;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t cl = v.candL[i];
    const uint32_t mi = v.candL_match[i];
    const uint32_t a = static_cast<uint32_t>(cl >> 32), b = static_cast<uint32_t>(cl);
    uint64_t s[kMaxVecWords];
#pragma unroll
    for (int w = 0; w < kMaxVecWords; ++w)
      s[w] = w < W ? v.qvec[0][w * v.qsize[0] + a] + v.qvec[2][w * v.qsize[2] + b] : 0;
    const unsigned long long rb = v.candR_off[mi], re = v.candR_off[mi + 1];
    unsigned long long checked = 0;
    for (unsigned long long j = rb; j < re; ++j) {
      const uint64_t cr = v.candR[j];
      const uint32_t c = static_cast<uint32_t>(cr >> 32), e = static_cast<uint32_t>(cr);
      bool ok = true;
#pragma unroll
      for (int w = 0; w < kMaxVecWords; ++w)
        if (w < W) ok &= (s[w] + v.qvec[1][w * v.qsize[1] + c] + v.qvec[3][w * v.qsize[3] + e]) == v.ic.dvec[w];
      ++checked;
      if (!ok) continue;
      uint64_t mask[2] = {0, 0};
      add_mask(mask, a, v.ic.col0[0]);
      add_mask(mask, c, v.ic.col0[1]);
      add_mask(mask, b, v.ic.col0[2]);
      add_mask(mask, e, v.ic.col0[3]);
      const unsigned long long slot = atomicAdd(v.sol_count, 1ull);
      if (slot < v.sol_cap) {
        v.sol[2 * slot] = mask[0];
        v.sol[2 * slot + 1] = mask[1];
      }
    }
    if (checked) atomicAdd(v.pairs_checked, checked);
  }
}

cudaError_t launch_verify(const VerifyDev &v, cudaStream_t s) {
  if (v.nL == 0) return cudaSuccess;
  uint64_t blocks = (v.nL + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  verify_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(v);
  return cudaGetLastError();
}

}  // namespace msp
