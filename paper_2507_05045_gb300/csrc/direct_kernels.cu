// Direct pass of libmsp (sm_103a): residue classes small enough that one
// thread block joins a whole class in shared memory, so no half-pair record
// is ever written to device memory.
//
// Split.  The columns are cut into a left half (L, the first ceil(n/2)) and a
// right half (R).  Each half is split again into an OUTER quarter of at most
// 2^9 subsets and an INNER quarter of up to 2^31 subsets: the four lists of
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
//   win_low/high_kernel, win_kernel  build the bucketed inner list of one
//                       instance: the low subsets (walked in Gray order) and
//                       the high subsets of the quarter, then the list by
//                       windows of classes, staged in shared memory;
//                       direct_inner_batch/offsets_kernel build those of
//                       every instance of a batch at once (one level).
//   direct_join_kernel  (direct_join.cu) the class joins in shared memory.
//   direct_verify_kernel one block per matched (class, key): finds every
//                       L pair (a, b) and R pair (c, e) with that key by
//                       scanning the class's inner buckets, and checks each
//                       of their combinations on all m rows (Algorithm 2's
//                       "if A x = d").
//   c1_dp_kernel        C1 = #{x : row_1 . x = d_1}, the number of row-1
//                       candidate pairs the solve rules on (subset-sum
//                       counting over row 1, 128-bit).
#include "direct_internal.cuh"

namespace msp {

namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr int kDT = kDirectThreads;       // threads per block of the inner and verify kernels

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

// Inner list of one instance, built by windows of classes.  The q inner
// columns split into h low and hq = min(q, 10) high ones.  The 2^h low
// subsets are bucketed by class at a coarse granularity of 2^gshift classes
// (a counting sort of at most 2^21 subsets).  Class r of the quarter holds
// the pairs (H, l) with kappa(H) + kappa(l) = r, so for each high subset H
// the classes of a window [w0, w0 + W) take the low subsets whose class
// lies in the cyclic interval [w0 - kappa(H), w0 - kappa(H) + W): a few
// coarse buckets, that is one contiguous run of the low list (two where the
// interval wraps).  One block per window counts its classes (first pass);
// given the bucket starts, it then places its subsets in a shared-memory
// stage and writes the window's range of the list with coalesced stores
// (second pass).  The random accesses all go to shared memory or to the low
// list, which stays in L2.
constexpr int kWinThreads = 512;

template <bool kScatter>
__global__ void win_low_kernel(InnerGen g, int c, uint64_t nchunks, int gshift, uint32_t *cnt_or_cur, uint4 *low) {
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < nchunks;
       t += (uint64_t)gridDim.x * blockDim.x) {
    walk_chunk(g, static_cast<uint32_t>(t << c), c, [&](uint32_t mask, uint32_t k, uint32_t r) {
      if constexpr (kScatter) {
        const uint32_t pos = atomicAdd(cnt_or_cur + (r >> gshift), 1u);
        low[pos] = make_uint4(k, mask, r, 0u);
      } else {
        atomicAdd(cnt_or_cur + (r >> gshift), 1u);
      }
    });
  }
}

// Key and class of every high subset H (columns h .. h + hq - 1).
__global__ void win_high_kernel(InnerGen g, int h, int hq, uint32_t *hkey, uint32_t *hcls) {
  const uint32_t H = blockIdx.x * blockDim.x + threadIdx.x;
  if (H >= (1u << hq)) return;
  uint32_t key = 0, cls = 0;
  for (uint32_t b = H; b; b &= b - 1) {
    const int j = h + __ffs(b) - 1;
    key += g.ck[j];
    cls += g.cc[j];
  }
  hkey[H] = g.neg ? 0u - key : key;
  hcls[H] = (g.neg ? 0u - cls : cls) & g.cmask;
}

// S1 for an outer quarter: one block per segment, one thread per subset,
// which sums the tables of its columns.
__global__ void __launch_bounds__(kOuterMax) direct_outer_kernel(const OuterSeg *segs) {
  const OuterSeg &g = segs[blockIdx.x];
  const uint32_t u = threadIdx.x;
  if (u >= (1u << g.q)) return;
  uint32_t key = 0, cls = 0;
  uint64_t v[4] = {0, 0, 0, 0};
  for (uint32_t b = u; b; b &= b - 1) {
    const int j = __ffs(b) - 1;
    key += g.ck[j];
    cls += g.cc[j];
#pragma unroll
    for (int w = 0; w < 4; ++w) v[w] += g.pc[j][w];
  }
  g.okey[u] = g.neg ? g.kd - key : key;
  g.ocls[u] = (g.neg ? g.cd - cls : cls) & g.cmask;
  g.omask[u] = u;
#pragma unroll
  for (int w = 0; w < 4; ++w) g.ovec[(size_t)u * 4 + w] = v[w];
}

template <bool kPlace>
__global__ void __launch_bounds__(kWinThreads) win_kernel(WinBuild w) {
  extern __shared__ __align__(16) uint8_t wsm[];
  uint2 *const stage = reinterpret_cast<uint2 *>(wsm);                  // [kWinCap] (place pass)
  uint32_t *const cur = reinterpret_cast<uint32_t *>(wsm + (kPlace ? sizeof(uint2) * kWinCap : 0));  // [W]
  const uint32_t W = 1u << w.logW;
  const uint32_t w0 = blockIdx.x << w.logW;
  uint32_t base = 0, total = 0;
  if (kPlace) {
    base = w.ioff[w0];
    total = w.ioff[w0 + W] - base;
  }
  for (uint32_t i = threadIdx.x; i < W; i += kWinThreads) cur[i] = kPlace ? w.ioff[w0 + i] - base : 0u;
  __syncthreads();
  const bool staged = total <= kWinCap;
  const bool whole = w.logW == w.B;  // one window: every low subset
  const uint32_t nH = 1u << w.hq;
  for (uint32_t H = threadIdx.x; H < nH; H += kWinThreads) {
    const uint32_t kH = w.hkey[H], cH = w.hcls[H];
    const uint32_t hm = H << w.h;
    uint32_t a0, a1, b0 = 0, b1 = 0;  // runs [a0, a1) and [b0, b1) of the low list
    if (whole) {
      a0 = 0;
      a1 = w.loff[w.nc];
    } else {
      const uint32_t st = (w0 - cH) & w.cmask;
      const uint32_t en = (st + W - 1u) & w.cmask;
      const uint32_t c1 = st >> w.gshift, c2 = en >> w.gshift;
      a0 = w.loff[c1];
      if (c2 >= c1) {
        a1 = w.loff[c2 + 1];
      } else {
        a1 = w.loff[w.nc];
        b1 = w.loff[c2 + 1];
      }
    }
    auto visit = [&](uint32_t i) {
      const uint4 e = w.low[i];
      const uint32_t d = (cH + e.z - w0) & w.cmask;
      if (d < W) {
        const uint32_t pos = atomicAdd(cur + d, 1u);
        if (kPlace) {
          const uint32_t key = kH + e.x, mask = hm | e.y;
          if (staged) {
            if (MSP_IN_BOUNDS(pos, kWinCap, 31u)) stage[pos] = make_uint2(key, mask);  // stage slot
          } else if (MSP_IN_BOUNDS(base + pos, 1ull << (w.h + w.hq), 32u)) {  // list position
            w.ikey[base + pos] = key;
            w.imask[base + pos] = mask;
          }
        }
      }
    };
#pragma unroll 4
    for (uint32_t i = a0; i < a1; ++i) visit(i);
    for (uint32_t i = b0; i < b1; ++i) visit(i);
  }
  __syncthreads();
  if (!kPlace) {
    for (uint32_t i = threadIdx.x; i < W; i += kWinThreads) w.cnt[w0 + i] = cur[i];
  } else if (staged) {
    for (uint32_t i = threadIdx.x; i < total; i += kWinThreads) {
      if (!MSP_IN_BOUNDS(base + i, 1ull << (w.h + w.hq), 33u)) continue;  // list position
      const uint2 v = stage[i];
      w.ikey[base + i] = v.x;
      w.imask[base + i] = v.y;
    }
  }
}

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
        if (!MSP_IN_BOUNDS(pos, 1ull << S.g.q, 34u)) return;  // list position
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




// -------------------------------------------------------------------------
// Recovery and exact verification of the matched (class, key) pairs.
// -------------------------------------------------------------------------
constexpr int kVT = 512;  // one thread per outer subset of each side
constexpr int kVCand = 512;



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
  const uint32_t key = v.match_key[blockIdx.x];
  const uint32_t tagged = v.match_cls[blockIdx.x];
  const uint32_t ii = tagged >> v.class_bits;
  const uint32_t r = tagged & v.cmask;
  const DirectVerifyInst &vi = v.inst[ii];
  if (threadIdx.x < 2) ncand[threadIdx.x] = 0;
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
    // eight inner keys of a side per step, loaded together (a bucket holds
    // about 16)
#pragma unroll
    for (int s = 0; s < 2; ++s)
      for (uint32_t j0 = b0[s]; j0 < b1[s]; j0 += 8) {
        uint32_t kk[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const bool in = j0 + u < b1[s] && MSP_IN_BOUNDS(j0 + u, vi.side[s].ni, 21u);  // bucket scan position
          kk[u] = in ? vi.side[s].ikey[j0 + u] : ~key;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (j0 + u < b1[s] && ka[s] + kk[u] == key) {
            const uint32_t slot = atomicAdd(&ncand[s], 1u);
            if (slot < kVCand) cand[s][slot] = make_uint2(static_cast<uint32_t>(a), j0 + u);
          }
      }
  }
  __syncthreads();
  const uint32_t nL = min(ncand[0], static_cast<uint32_t>(kVCand));
  const uint32_t nR = min(ncand[1], static_cast<uint32_t>(kVCand));
  if (threadIdx.x == 0) {
    if (ncand[0] > kVCand || ncand[1] > kVCand) atomicOr(v.overflow, 1u);
    // spread over kVerifyPairSlots counters: one shared address would
    // serialise the atomics of all blocks
    atomicAdd(v.pairs + (blockIdx.x % kVerifyPairSlots), (unsigned long long)nL * nR);
  }
  const uint32_t np = nL * nR;
  for (uint32_t pi = threadIdx.x; pi < np; pi += kVT) {
    const uint2 l = cand[0][pi / nR], rr = cand[1][pi % nR];
    if (!MSP_IN_BOUNDS(l.y, vi.side[0].ni, 22u) || !MSP_IN_BOUNDS(rr.y, vi.side[1].ni, 23u) ||
        !MSP_IN_BOUNDS(l.x, static_cast<uint32_t>(vi.side[0].no), 24u) ||
        !MSP_IN_BOUNDS(rr.x, static_cast<uint32_t>(vi.side[1].no), 25u))
      continue;  // candidate positions inside the lists
    uint64_t vec[4];
    for (int w = 0; w < 4; ++w) vec[w] = vi.ovec[0][l.x * 4 + w] + vi.ovec[1][rr.x * 4 + w];
    const uint32_t mL = vi.imask[0][l.y], mR = vi.imask[1][rr.y];
    // the packed inner columns are read where a pair needs them (about one
    // pair per match; the two column tables stay in cache)
    for (uint32_t b = mL; b; b &= b - 1) {
      const int j = __ffs(b) - 1;
      for (int w = 0; w < 4; ++w) vec[w] += __ldg(vi.icol[0] + j * 4 + w);
    }
    for (uint32_t b = mR; b; b &= b - 1) {
      const int j = __ffs(b) - 1;
      for (int w = 0; w < 4; ++w) vec[w] += __ldg(vi.icol[1] + j * 4 + w);
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

}  // namespace

cudaError_t launch_win_low(const InnerGen &g, int gshift, uint32_t *cnt_or_cur, uint4 *low, cudaStream_t s) {
  const int c = g.q < kGenChunk ? g.q : kGenChunk;
  const uint64_t nchunks = (uint64_t(1) << g.q) >> c;
  const uint64_t want = (nchunks + 255) / 256;
  const unsigned blocks = static_cast<unsigned>(want < (1u << 20) ? want : (1u << 20));
  if (low)
    win_low_kernel<true><<<blocks, 256, 0, s>>>(g, c, nchunks, gshift, cnt_or_cur, low);
  else
    win_low_kernel<false><<<blocks, 256, 0, s>>>(g, c, nchunks, gshift, cnt_or_cur, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_win_high(const InnerGen &g, int h, int hq, uint32_t *hkey, uint32_t *hcls, cudaStream_t s) {
  const unsigned n = 1u << hq;
  win_high_kernel<<<(n + 255) / 256, 256, 0, s>>>(g, h, hq, hkey, hcls);
  return cudaGetLastError();
}

cudaError_t launch_direct_outer(const OuterSeg *segs, int nseg, cudaStream_t s) {
  if (nseg < 1) return cudaSuccess;
  static_assert((1 << kOuterColsMax) <= kOuterMax, "one thread per outer subset");
  direct_outer_kernel<<<nseg, kOuterMax, 0, s>>>(segs);
  return cudaGetLastError();
}

cudaError_t launch_win(const WinBuild &w, bool place, cudaStream_t s) {
  if (w.logW > w.B || w.B > 31 || w.h + w.hq > kInnerMax) return cudaErrorInvalidValue;
  const unsigned windows = 1u << (w.B - w.logW);
  const size_t cur = sizeof(uint32_t) << w.logW;
  if (place) {
    static bool attr = false;
    const size_t smem = sizeof(uint2) * kWinCap + (sizeof(uint32_t) << kWinBits);
    if (!attr) {
      const cudaError_t e =
          cudaFuncSetAttribute(win_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
      if (e != cudaSuccess) return e;
      attr = true;
    }
    win_kernel<true><<<windows, kWinThreads, sizeof(uint2) * kWinCap + cur, s>>>(w);
  } else {
    win_kernel<false><<<windows, kWinThreads, cur, s>>>(w);
  }
  return cudaGetLastError();
}

cudaError_t launch_direct_inner_batch(const InnerSeg *segs, int nseg, int q, bool scatter, cudaStream_t s) {
  const int c = q < kGenChunk ? q : kGenChunk;
  const uint64_t per = (uint64_t(1) << q) >> c;
  const uint64_t total = per * static_cast<uint64_t>(nseg);
  const uint64_t want = (total + 255) / 256;
  const unsigned blocks = static_cast<unsigned>(want < (1u << 20) ? want : (1u << 20));
  if (scatter)
    direct_inner_batch_kernel<true><<<blocks, 256, 0, s>>>(segs, c, per, total);
  else
    direct_inner_batch_kernel<false><<<blocks, 256, 0, s>>>(segs, c, per, total);
  return cudaGetLastError();
}

cudaError_t launch_direct_inner_offsets(const InnerSeg *segs, int nseg, uint32_t M, cudaStream_t s) {
  direct_inner_offsets_kernel<<<static_cast<unsigned>(nseg), 1024, 0, s>>>(segs, M);
  return cudaGetLastError();
}

cudaError_t launch_direct_verify(const DirectVerify &v, unsigned nmatch, cudaStream_t s) {
  direct_verify_kernel<<<nmatch, kVT, 0, s>>>(v);
  return cudaGetLastError();
}

cudaError_t launch_c1_dp(const int32_t *a1, int n, int d1, void *buf, unsigned long long *out, cudaStream_t s) {
  c1_dp_kernel<<<1, 1024, 0, s>>>(a1, n, d1, static_cast<unsigned __int128 *>(buf), out);
  return cudaGetLastError();
}

}  // namespace msp
