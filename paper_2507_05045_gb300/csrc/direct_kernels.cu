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
//   direct_inner_count/scatter_kernel  build the bucketed inner lists
//                       (counting sort of all 2^qi subsets by class; each
//                       thread walks a chunk of subsets in Gray order);
//                       direct_inner_batch/offsets_kernel do the same for
//                       every instance of a batch at once.
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
    // eight inner keys of a side per step, loaded together (a bucket holds
    // about 16)
#pragma unroll
    for (int s = 0; s < 2; ++s)
      for (uint32_t j0 = b0[s]; j0 < b1[s]; j0 += 8) {
        uint32_t kk[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) kk[u] = j0 + u < b1[s] ? vi.side[s].ikey[j0 + u] : ~key;
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

}  // namespace

cudaError_t launch_direct_inner(const InnerGen &g, uint32_t *cnt_or_cur, uint32_t *ikey, uint32_t *imask,
                                cudaStream_t s) {
  const int c = g.q < kGenChunk ? g.q : kGenChunk;
  const uint64_t nchunks = (uint64_t(1) << g.q) >> c;
  const uint64_t want = (nchunks + 255) / 256;
  const unsigned blocks = static_cast<unsigned>(want < (1u << 20) ? want : (1u << 20));
  if (ikey)
    direct_inner_scatter_kernel<<<blocks, 256, 0, s>>>(g, c, nchunks, cnt_or_cur, ikey, imask);
  else
    direct_inner_count_kernel<<<blocks, 256, 0, s>>>(g, c, nchunks, cnt_or_cur);
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
