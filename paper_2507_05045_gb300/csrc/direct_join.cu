// Class joins of the direct pass (sm_103a).  Persistent blocks of 512
// threads, two per SM, take work items of consecutive residue classes (of
// any instance of the launch) from a counter.  Per class, each warp owns one
// group of 32 outer subsets per side; it expands their records (the runs of
// consecutive keys of their inner buckets) and hands them, four per lane at a
// time, to the table code:
//   left keys set a bit of a shared filter and take a slot of their home
//   bucket (8 slots) through its counter, moving on to later buckets
//   through a per-warp queue when it is full;
//   after a block barrier, right keys test the filter, and the few that pass
//   (about 6 %) are looked up in the buckets through the queue; a matched
//   (class, key) is claimed once per slot and appended to a device list.
// A class whose left side exceeds one table fill is joined in several
// fills, each probed by every right key.  No record is written to device
// memory.
#include "direct_internal.cuh"

namespace msp {

namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr int kDT = kDirectThreads;       // threads per join block
constexpr int kDW = kDT / 32;             // warps per join block

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

constexpr int kQueue = 64;  // deferred keys per warp

// Shared join structures of a block, for a table of 2^TB slots:
//   T     2^TB key slots in buckets of 8 (bucket = top TB - 3 key bits);
//   C     one 32-bit fill counter per bucket;
//   F     a filter of 2^(TB + 3) bits (bit = top TB + 3 key bits) set for
//         every left key, so that most right keys are settled by one load;
//   claim one bit per slot: the slot's key was already reported.
// T is never cleared: a bucket's slots past its counter are not read.
__host__ __device__ constexpr uint32_t tab_words(int TB) { return 1u << TB; }
__host__ __device__ constexpr uint32_t cnt_words(int TB) { return 1u << (TB - 3); }
__host__ __device__ constexpr uint32_t filt_words(int TB) { return 1u << (TB - 2); }
__host__ __device__ constexpr uint32_t claim_words(int TB) { return 1u << (TB - 5); }

size_t direct_smem_bytes(int TB, int noL, int noR) {
  (void)noL;
  (void)noR;
  return (size_t)4 * (tab_words(TB) + cnt_words(TB) + filt_words(TB) + claim_words(TB))
         + (size_t)kDW * 32 * 8         // per-warp element table
         + (size_t)kDW * 32 * 4         // per-warp start bitmaps
         + (size_t)kDW * 32 * 4         // per-warp word bases
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
// inner keys of a batch are loaded together, so their latencies overlap.
// Record k belongs to the last nonempty subset whose first record is <= k;
// a bitmap marks the first records (1024 records per segment, one word per
// lane, with the count of first records before each word beside it) and a
// compacted per-warp table holds (start - first record, ka).
constexpr int kBatch = 4;
static_assert(kBatch == 4, "a batch reads its bitmap words and bases as one uint4 each");

template <typename F>
__device__ __forceinline__ void group_records(uint32_t st, uint32_t len, uint32_t ka,
                                              const uint32_t *__restrict__ ikey, uint32_t ni, uint2 *et_w,
                                              uint32_t *bm_w,
                                              uint32_t *wb_w, uint32_t lo, uint32_t hi, F &&f) {
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
    const uint32_t before = __popc(__ballot_sync(kFull, len != 0 && pre < S));
    const uint32_t pc = __popc(myw);
    uint32_t wi = pc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, wi, o);
      if (ln >= static_cast<uint32_t>(o)) wi += y;
    }
    const uint32_t wbase = before + wi - pc;
    wb_w[ln] = wbase;
    __syncwarp();
    const uint32_t send = min(ke, S + 1024u);
    // inner key and outer key of each record of the batch at i0
    auto fetch = [&](uint32_t i0, uint32_t (&raw)[kBatch], uint32_t (&ko)[kBatch], uint32_t &okm) {
      okm = 0u;
      // i0 - S is a multiple of 32 kBatch: the bitmap words and their bases
      // of the batch's kBatch = 4 rows of 32 records in two broadcast loads
      const uint32_t w0 = (i0 - S) >> 5;
      const uint4 wv = *reinterpret_cast<const uint4 *>(bm_w + w0);
      const uint4 bv = *reinterpret_cast<const uint4 *>(wb_w + w0);
      const uint32_t wa[kBatch] = {wv.x, wv.y, wv.z, wv.w};
      const uint32_t ba[kBatch] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int b = 0; b < kBatch; ++b) {
        const uint32_t word = wa[b];
        const uint32_t base = ba[b];
        const uint32_t k = i0 + 32u * b + ln;
        bool ok = k >= lo && k < send;
        const uint32_t c = base + __popc(word & lemask) - 1u;
        if (ok && !MSP_IN_BOUNDS(c, 32u, 11u)) ok = false;  // compacted subset of the group
        const uint2 e = et_w[ok ? c : 0u];
        // lanes outside the range read inner element 0: every address
        // formed here lies inside the inner list
        uint32_t pos = ok ? e.x + k : 0u;
        if (ok && !MSP_IN_BOUNDS(pos, ni, 12u)) {  // inner position of the record
          ok = false;
          pos = 0u;
        }
        raw[b] = __ldg(ikey + pos);
        ko[b] = e.y;
        okm |= static_cast<uint32_t>(ok) << b;
      }
    };
    for (uint32_t i0 = S; i0 < send; i0 += 32u * kBatch) {
      uint32_t rc[kBatch], kc[kBatch], okc, key[kBatch];
      fetch(i0, rc, kc, okc);
#pragma unroll
      for (int b = 0; b < kBatch; ++b) key[b] = kc[b] + rc[b];
      f(okc, key);
    }
    __syncwarp();  // every lane has read this segment's words
    bm_w[ln] = 0u;
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
  uint32_t *const wbb = wbm + kDW * 32;     // [kDW][32] record counts before each bitmap word
  uint32_t *const wq = wbb + kDW * 32;      // [kDW][kQueue]
  uint32_t *const wtot = wq + kDW * kQueue;
  const int noL = p.no[0], noR = p.no[1];
  // each warp's record totals of a class (left, right), double-buffered by
  // class parity: class i writes slot i & 1 before its first barrier and
  // every warp sums the slot after it, with no shared atomics
  __shared__ uint2 s_wsum[2][kDW];
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
    s_bad[threadIdx.x] = 0;
  }
  uint2 *const et_w = et + wp * 32;
  uint32_t *const bm_w = wbm + wp * 32;
  uint32_t *const wb_w = wbb + wp * 32;
  uint32_t *const q_w = wq + wp * kQueue;
  const uint32_t ltmask = (1u << ln) - 1u;
  uint32_t qn = 0;  // deferred keys of this warp (warp-uniform)
  // Count-claimed slot: the previous fill of bucket b.
  auto take_slot = [&](uint32_t b) -> uint32_t { return atomicAdd(C + b, 1u); };
  auto count_of = [&](uint32_t b) -> uint32_t { return C[b]; };
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
  uint32_t kaL = 0, kaR = 0, clL = 0, clR = 0, niL = 0, niR = 0;
  uint32_t cur_inst = 0xffffffffu;
  uint32_t pfL0 = 0, pfL1 = 0, pfR0 = 0, pfR1 = 0;
  // carry: class r follows the previous class of the same work item, so a
  // bucket starts where the previous one (r - 1) ended, unless the bucket
  // index wrapped to 0
  auto load_bounds = [&](uint32_t r, bool carry) {
    if (el < noL) {
      const uint32_t w = (r - clL) & cmask;
      pfL0 = carry && w != 0u ? pfL1 : ioffL[w];
      pfL1 = ioffL[w + 1];
    } else {
      pfL0 = pfL1 = 0u;
    }
    if (el < noR) {
      const uint32_t w = (r - clR) & cmask;
      pfR0 = carry && w != 0u ? pfR1 : ioffR[w];
      pfR1 = ioffR[w + 1];
    } else {
      pfR0 = pfR1 = 0u;
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
      niL = s_inst.side[0].ni;
      niR = s_inst.side[1].ni;
      kaL = el < noL ? s_inst.side[0].okey[el] : 0u;
      clL = el < noL ? s_inst.side[0].ocls[el] : 0u;
      kaR = el < noR ? s_inst.side[1].okey[el] : 0u;
      clR = el < noR ? s_inst.side[1].ocls[el] : 0u;
    }
    const uint32_t tag = ii << p.class_bits;
    const uint32_t rb = (item - ii * per_inst) * p.chunk, re = min(p.nclass, rb + p.chunk);
    for (uint32_t ri = rb; ri < re; ++ri, par ^= 1u) {
      const uint32_t r = (p.c0 + ri) & cmask;
      // ---- bucket of this warp's outer subsets (lane = subset) ----
      load_bounds(r, ri > rb);
      const uint32_t stL = pfL0, lnL = pfL1 - pfL0, stR = pfR0, lnR = pfR1 - pfR0;
      const bool big = __any_sync(kFull, lnL >= (1u << 24) || lnR >= (1u << 24));
      // a warp's 32 buckets, each clamped to 2^24 (a larger one skips the
      // class), stay below 2^29 records
      const uint32_t sumL = __reduce_add_sync(kFull, min(lnL, 1u << 24));
      const uint32_t sumR = __reduce_add_sync(kFull, min(lnR, 1u << 24));
      if (ln == 0) {
        s_wsum[par][wp] = make_uint2(sumL, sumR);
        wtot[wp] = sumL;
        if (big) {
          atomicOr(&s_bad[par], 1u);
          atomicOr(p.error, 1u);
        }
      }
      __syncthreads();
      // class totals: lane w < kDW takes warp w's totals
      unsigned long long TL = 0, TR = 0;
      if (ln < static_cast<uint32_t>(kDW)) {
        const uint2 t = s_wsum[par][ln];
        TL = t.x;
        TR = t.y;
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        TL += __shfl_xor_sync(kFull, TL, o);
        TR += __shfl_xor_sync(kFull, TR, o);
      }
      // a class past 2^31 records on a side, or a bucket past 2^24, is beyond
      // this kernel: it is skipped and the host, seeing the error flag, solves
      // the instance on another path
      const bool skip = s_bad[par] != 0u || TL >= (1ull << 31) || TR >= (1ull << 31);
      if (skip && threadIdx.x == 0) atomicOr(p.error, 1u);
      if (threadIdx.x == 0) {
        my_records += TL + TR;
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
          group_records(stL, lnL, kaL, ikeyL, niL, et_w, bm_w, wb_w, lo, hi,
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
          group_records(stR, lnR, kaR, ikeyR, niR, et_w, bm_w, wb_w, 0u, 0xffffffffu,
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

cudaError_t launch_direct_join_impl(int TB, const DirectPass &p, cudaStream_t s) {
  switch (TB) {
    case 12: return launch_direct_join_tb<12>(p, s);
    case 13: return launch_direct_join_tb<13>(p, s);
    case 14: return launch_direct_join_tb<14>(p, s);
    case 15: return launch_direct_join_tb<15>(p, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_direct_join(int TB, const DirectPass &p, cudaStream_t s) {
  return launch_direct_join_impl(TB, p, s);
}

}  // namespace msp
