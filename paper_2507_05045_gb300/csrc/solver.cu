// Host side of libmsp: validation, the pass planner and the C ABI of
// include/msp.h.  Every arithmetic step of a solve runs in the kernels of
// kernels.cu; the host only plans, allocates, launches and collects.
#include "msp_internal.cuh"
#include "../../include/msp.h"
#include "host_internal.h"

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

namespace msp {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}

// splitmix64 (Steele, Lea, Flood 2014) for the fixed key weights.
static uint64_t splitmix(uint64_t &s) {
  s += 0x9E3779B97F4A7C15ull;
  uint64_t z = s;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct Plan {
  int m, n, W;
  int q[4], col0[4];
  int lgL, lgR;        // log2 |L|, |R|
  int B, t, D, S;
  uint32_t c_row[kMaxClassRows];
  uint64_t w_row[kMaxRows];
};

// Quarters: sizes ceil(n/4) for the first n mod 4 quarters, floor(n/4) for
// the rest; L pairs the largest quarter Q1 with Q3, R pairs Q2 with Q4.
Plan make_plan(int m, int n) {
  Plan p{};
  p.m = m;
  p.n = n;
  p.W = (m + 3) / 4;
  int c = 0;
  for (int k = 0; k < 4; ++k) {
    p.q[k] = n / 4 + (k < n % 4 ? 1 : 0);
    p.col0[k] = c;
    c += p.q[k];
  }
  p.lgL = p.q[0] + p.q[2];
  p.lgR = p.q[1] + p.q[3];
  const int lgmax = std::max(p.lgL, p.lgR);
  // about 2^23 records per class and side; partitions of about 2^12.
  p.B = std::min(22, std::max(0, lgmax - 23));
  p.t = p.B <= 8 ? 1 : (p.B <= 14 ? 2 : 3);
  p.t = std::min(p.t, m);
  p.D = std::min(12, std::max(0, lgmax - p.B - 12));
  p.S = 10;  // 1024 shared-memory buckets per side (about 4 keys each)
  uint64_t s = 0x2507050450000001ull;
  p.c_row[0] = 1;
  for (int i = 1; i < kMaxClassRows; ++i) p.c_row[i] = static_cast<uint32_t>(splitmix(s)) | 1u;
  for (int i = 0; i < kMaxRows; ++i) p.w_row[i] = splitmix(s) | 1ull;
  return p;
}

}  // namespace msp

using namespace msp;

namespace {

struct DevAlloc {
  cudaStream_t s;
  std::vector<void *> ptrs;
  size_t bytes = 0, peak = 0;
  explicit DevAlloc(cudaStream_t st) : s(st) {}
  template <typename T>
  cudaError_t get(T **p, size_t count) {
    void *q = nullptr;
    const size_t b = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMallocAsync(&q, b, s);
    if (e != cudaSuccess) return e;
    ptrs.push_back(q);
    bytes += b;
    peak = std::max(peak, bytes);
    *p = static_cast<T *>(q);
    return cudaSuccess;
  }
  void free1(void *q, size_t b) {
    for (auto &x : ptrs)
      if (x == q) {
        cudaFreeAsync(q, s);
        x = nullptr;
        bytes -= b;
        return;
      }
  }
  void release() {
    for (void *q : ptrs)
      if (q) cudaFreeAsync(q, s);
    ptrs.clear();
    bytes = 0;
  }
  ~DevAlloc() { release(); }
};

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      return fail(e_ == cudaErrorMemoryAllocation ? MSP_ENOMEM : MSP_ECUDA,           \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                \
    }                                                                                 \
  } while (0)

int validate(const int32_t *A, const int32_t *d, int m, int n) {
  if (!A || !d) return fail(MSP_EINVAL, "A and d must be non-null");
  if (m < 1 || m > kMaxRows) return fail(MSP_ERANGE, "m must lie in [1, 16]");
  if (n < 1 || n > kMaxN) return fail(MSP_ERANGE, "n must lie in [1, 100]");
  for (int i = 0; i < m; ++i) {
    if (d[i] < 0) return fail(MSP_EINVAL, "d has a negative entry");
    int64_t s = 0;
    for (int j = 0; j < n; ++j) {
      if (A[(size_t)i * n + j] < 0) return fail(MSP_EINVAL, "A has a negative entry");
      s += A[(size_t)i * n + j];
    }
    if (s >= 65536) return fail(MSP_ERANGE, "a row sum reaches 2^16");
  }
  return MSP_OK;
}

uint64_t key_of(const Plan &p, const int64_t *v) {
  uint64_t k = 0;
  for (int i = 0; i < p.m; ++i) k += p.w_row[i] * static_cast<uint64_t>(v[i]);
  return k;
}

uint32_t class_of(const Plan &p, const int64_t *v) {
  uint32_t c = 0;
  for (int i = 0; i < p.t; ++i) c += p.c_row[i] * static_cast<uint32_t>(v[i]);
  return p.B ? (c & ((1u << p.B) - 1u)) : 0u;
}

struct SolveResult {
  std::vector<uint64_t> masks;  // [count][2]
};

// The solve proper.  `out` receives unsorted solution masks (two words each).
int solve_impl(msp_instance *inst, SolveResult *res) {
  const int m = inst->m, n = inst->n;
  const Plan p = make_plan(m, n);
  cudaStream_t s = inst->stream;
  msp_stats &st = inst->stats;
  st = msp_stats{};
  st.m = m;
  st.n = n;
  for (int k = 0; k < 4; ++k) st.quarter[k] = p.q[k];
  st.class_bits = p.B;
  st.class_rows = p.t;
  st.digit_bits = p.D;
  st.records_left = 1ull << p.lgL;
  st.records_right = 1ull << p.lgR;

  // Infeasible right-hand side: some d_i exceeds its row sum.
  std::vector<int64_t> rowsum(m, 0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) rowsum[i] += inst->A[(size_t)i * n + j];
  for (int i = 0; i < m; ++i)
    if (inst->d[i] > rowsum[i]) return MSP_OK;

  // ---- S0: packed columns, key and class of every column, constants ----
  InstanceConst ic{};
  ic.m = m;
  ic.n = n;
  ic.W = p.W;
  for (int k = 0; k < 4; ++k) {
    ic.q[k] = p.q[k];
    ic.col0[k] = p.col0[k];
  }
  for (int i = 0; i < kMaxRows; ++i) ic.w_row[i] = p.w_row[i];
  for (int i = 0; i < kMaxClassRows; ++i) ic.c_row[i] = p.c_row[i];
  ic.t_rows = p.t;
  ic.class_bits = p.B;
  std::vector<uint64_t> pcol((size_t)n * kMaxVecWords, 0), kcol(n);
  std::vector<uint32_t> ccol(n);
  std::vector<int64_t> col(m);
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < m; ++i) {
      col[i] = inst->A[(size_t)i * n + j];
      pcol[(size_t)j * kMaxVecWords + i / 4] |= static_cast<uint64_t>(col[i]) << (16 * (i % 4));
    }
    kcol[j] = key_of(p, col.data());
    uint32_t c = 0;
    for (int i = 0; i < p.t; ++i) c += p.c_row[i] * static_cast<uint32_t>(col[i]);
    ccol[j] = c;
  }
  std::vector<int64_t> dv(m);
  for (int i = 0; i < m; ++i) {
    dv[i] = inst->d[i];
    ic.dvec[i / 4] |= static_cast<uint64_t>(dv[i]) << (16 * (i % 4));
  }
  ic.kd = key_of(p, dv.data());
  ic.cd = class_of(p, dv.data());

  const uint32_t M = 1u << p.B;
  const uint32_t cmask = M - 1u;

  DevAlloc da(s);
  uint64_t *d_pcol, *d_kcol;
  uint32_t *d_ccol;
  CK(da.get(&d_pcol, pcol.size()));
  CK(da.get(&d_kcol, kcol.size()));
  CK(da.get(&d_ccol, ccol.size()));
  CK(cudaMemcpyAsync(d_pcol, pcol.data(), pcol.size() * 8, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_kcol, kcol.data(), kcol.size() * 8, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_ccol, ccol.data(), ccol.size() * 4, cudaMemcpyHostToDevice, s));

  // ---- S1: quarter lists ----
  QuarterDev qd[4];
  for (int k = 0; k < 4; ++k) {
    qd[k].q = p.q[k];
    qd[k].size = int64_t(1) << p.q[k];
    CK(da.get(&qd[k].vec, (size_t)p.W * qd[k].size));
    CK(da.get(&qd[k].key, qd[k].size));
    CK(da.get(&qd[k].cls, qd[k].size));
    CK(da.get(&qd[k].v1, qd[k].size));
    CK(launch_gray(ic, d_pcol, d_kcol, d_ccol, qd[k], p.col0[k], s));
  }

  // ---- S2: bucket the four lists by (transformed) class ----
  // list 0: Q1 (L outer), 1: Q3 (L inner), 2: Q2' (R outer), 3: Q4' (R inner)
  const int qk[4] = {0, 2, 1, 3};
  const int64_t mul[4] = {1, 1, -1, -1};
  const uint64_t kadd[4] = {0, 0, ic.kd, 0};
  const uint32_t cadd[4] = {0, 0, ic.cd, 0};
  BucketDev bd[4];
  uint32_t *d_hist, *d_cursor, *d_scantmp;
  CK(da.get(&d_hist, M));
  CK(da.get(&d_cursor, (size_t)M + 1));
  CK(da.get(&d_scantmp, ((size_t)M + 1 + 4095) / 4096 + 1));
  for (int l = 0; l < 4; ++l) {
    const QuarterDev &q = qd[qk[l]];
    bd[l].size = q.size;
    CK(da.get(&bd[l].key, q.size));
    CK(da.get(&bd[l].cls, q.size));
    CK(da.get(&bd[l].idx, q.size));
    CK(da.get(&bd[l].off, (size_t)M + 1));
    CK(cudaMemsetAsync(d_hist, 0, sizeof(uint32_t) * M, s));
    CK(launch_count_classes(q.cls, q.size, static_cast<uint32_t>(mul[l]), cadd[l], cmask, d_hist, s));
    CK(launch_scan_u32(d_hist, bd[l].off, M, d_scantmp, s));
    CK(cudaMemcpyAsync(d_cursor, bd[l].off, sizeof(uint32_t) * M, cudaMemcpyDeviceToDevice, s));
    CK(launch_bucket_scatter(q, mul[l], kadd[l], cadd[l], cmask, d_cursor, bd[l], s));
  }

  // ---- row-1 candidate count C1 (the metric's unit of work) ----
  {
    int64_t qsum[4] = {0, 0, 0, 0};
    for (int k = 0; k < 4; ++k)
      for (int j = 0; j < p.q[k]; ++j) qsum[k] += inst->A[p.col0[k] + j];
    const int len13 = static_cast<int>(std::max(qsum[0], qsum[2]) + 1);
    const int len24 = static_cast<int>(std::max(qsum[1], qsum[3]) + 1);
    const int lenl = 2 * len13 - 1, lenr = 2 * len24 - 1;
    unsigned long long *h[4], *hl, *hr, *c1;
    for (int k = 0; k < 4; ++k) {
      const int len = (k == 0 || k == 2) ? len13 : len24;
      CK(da.get(&h[k], len));
      CK(cudaMemsetAsync(h[k], 0, sizeof(unsigned long long) * len, s));
      CK(launch_v1_hist(qd[k].v1, qd[k].size, h[k], s));
    }
    CK(da.get(&hl, lenl));
    CK(da.get(&hr, lenr));
    CK(da.get(&c1, 2));
    CK(launch_row1_candidates(h[0], h[2], len13, h[1], h[3], len24, hl, hr, lenl, lenr, inst->d[0], c1, s));
    unsigned long long c1h[2];
    CK(cudaMemcpyAsync(c1h, c1, sizeof(c1h), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    st.row1_candidates_lo = c1h[0];
    st.row1_candidates_hi = c1h[1];
  }

  // ---- pass setup ----
  PassDev pd{};
  pd.cmask = cmask;
  pd.D = p.D;
  pd.S = p.S;
  const int nd = 1 << p.D;
  for (int side = 0; side < 2; ++side) {
    const BucketDev &o = bd[side == 0 ? 0 : 2];
    const BucketDev &in = bd[side == 0 ? 1 : 3];
    SideGen &g = pd.side[side];
    g.okey = o.key;
    g.ocls = o.cls;
    g.osize = o.size;
    g.ikey = in.key;
    g.ioff = in.off;
    const int64_t per_bucket = std::max<int64_t>(1, in.size / M);
    g.slice_outer = std::max<int64_t>(1, (int64_t(1) << 19) / per_bucket);
    g.slices = static_cast<int>((o.size + g.slice_outer - 1) / g.slice_outer);
  }
  // memory budget
  size_t free_b = 0, total_b = 0;
  CK(cudaMemGetInfo(&free_b, &total_b));
  size_t budget = inst->budget ? inst->budget : static_cast<size_t>(0.85 * free_b);
  budget = std::min(budget, static_cast<size_t>(0.92 * free_b));
  const double est_class[2] = {std::ldexp(1.0, p.lgL - p.B), std::ldexp(1.0, p.lgR - p.B)};
  const size_t per_class_meta =
      (size_t)nd * (sizeof(uint64_t) + sizeof(uint32_t)) * 2 +
      (size_t)nd * sizeof(uint32_t) * (pd.side[0].slices + pd.side[1].slices) + 64;
  const double per_class_bytes = (est_class[0] + est_class[1]) * 8.0 * 1.08 + per_class_meta;
  const size_t fixed_reserve = (size_t)64 << 20;  // matches, lists of oversize partitions
  if (budget < fixed_reserve + per_class_bytes)
    return fail(MSP_ENOMEM, "memory budget too small for one residue class");
  int max_classes = static_cast<int>(std::min<double>(
      M, std::floor((double)(budget - fixed_reserve) / per_class_bytes)));
  max_classes = std::max(1, std::min(max_classes, 1 << 16));
  uint64_t rec_cap[2] = {
      static_cast<uint64_t>(std::min<double>(std::ldexp(1.0, p.lgL), est_class[0] * 1.08 * max_classes + 4096)),
      static_cast<uint64_t>(std::min<double>(std::ldexp(1.0, p.lgR), est_class[1] * 1.08 * max_classes + 4096))};
  for (int side = 0; side < 2; ++side) {
    CK(da.get(&pd.cnt[side], (size_t)max_classes * pd.side[side].slices * nd));
    CK(da.get(&pd.segstart[side], (size_t)max_classes * nd));
    CK(da.get(&pd.seglen[side], (size_t)max_classes * nd));
    CK(da.get(&pd.classtot[side], (size_t)max_classes));
    CK(da.get(&pd.classbase[side], (size_t)max_classes));
    CK(da.get(&pd.rec[side], rec_cap[side]));
  }
  pd.match_cap = 1u << 20;
  CK(da.get(&pd.match_key, pd.match_cap));
  CK(da.get(&pd.match_cls, pd.match_cap));
  CK(da.get(&pd.match_count, 1));
  CK(cudaMemsetAsync(pd.match_count, 0, sizeof(unsigned long long), s));
  pd.big_cap = static_cast<uint32_t>(std::min<uint64_t>((uint64_t)max_classes * nd, 1u << 24));
  CK(da.get(&pd.big_list, pd.big_cap));
  CK(da.get(&pd.big_count, 1));

  std::vector<uint64_t> tot_h(2 * (size_t)max_classes), base_h(2 * (size_t)max_classes);
  unsigned int big_h = 0;
  uint64_t oversize = 0;
  int passes = 0;
  for (uint32_t c0 = 0; c0 < M;) {
    if (inst->cancel && *inst->cancel) return fail(MSP_ECANCELED, "request canceled");
    pd.c0 = static_cast<int>(c0);
    pd.nclass = static_cast<int>(std::min<uint64_t>(max_classes, M - c0));
    CK(launch_gen_count(pd, s));
    CK(launch_counts_to_offsets(pd, s));
    CK(cudaMemcpyAsync(tot_h.data(), pd.classtot[0], sizeof(uint64_t) * pd.nclass, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(tot_h.data() + max_classes, pd.classtot[1], sizeof(uint64_t) * pd.nclass,
                       cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // the longest prefix of classes that fits both record buffers
    uint64_t acc[2] = {0, 0};
    int run = 0;
    for (int c = 0; c < pd.nclass; ++c) {
      const uint64_t a0 = tot_h[c], a1 = tot_h[max_classes + c];
      if (acc[0] + a0 > rec_cap[0] || acc[1] + a1 > rec_cap[1]) break;
      if (a0 >= (1ull << 31) || a1 >= (1ull << 31)) break;
      base_h[c] = acc[0];
      base_h[max_classes + c] = acc[1];
      acc[0] += a0;
      acc[1] += a1;
      ++run;
    }
    if (run == 0) {
      // A class larger than the buffers (skewed class sizes): grow them to
      // hold it if the budget allows, then retry the pass.
      const uint64_t need0 = tot_h[0], need1 = tot_h[max_classes];
      const double need_bytes = 8.0 * (double)(need0 + need1) + (double)da.bytes -
                                8.0 * (double)(rec_cap[0] + rec_cap[1]);
      if (need0 >= (1ull << 31) || need1 >= (1ull << 31) || need_bytes > (double)budget)
        return fail(MSP_ENOMEM, "one residue class does not fit the memory budget");
      for (int side = 0; side < 2; ++side) {
        const uint64_t need = side ? need1 : need0;
        if (need <= rec_cap[side]) continue;
        da.free1(pd.rec[side], sizeof(uint64_t) * rec_cap[side]);
        rec_cap[side] = need;
        CK(da.get(&pd.rec[side], rec_cap[side]));
      }
      continue;
    }
    CK(cudaMemcpyAsync(pd.classbase[0], base_h.data(), sizeof(uint64_t) * run, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(pd.classbase[1], base_h.data() + max_classes, sizeof(uint64_t) * run,
                       cudaMemcpyHostToDevice, s));
    CK(launch_gen_scatter(pd, run, s));
    CK(cudaMemsetAsync(pd.big_count, 0, sizeof(unsigned int), s));
    CK(launch_join(pd, run, s));
    CK(launch_join_big(pd, run, s));
    CK(cudaMemcpyAsync(&big_h, pd.big_count, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    oversize += big_h;
    if (big_h > pd.big_cap) return fail(MSP_EOVERFLOW, "too many oversize partitions in one pass");
    c0 += static_cast<uint32_t>(run);
    ++passes;
  }
  st.passes = passes;
  st.oversize_segments = oversize;

  unsigned long long nmatch = 0;
  CK(cudaMemcpyAsync(&nmatch, pd.match_count, sizeof(nmatch), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  st.key_matches = nmatch;
  if (nmatch > pd.match_cap) return fail(MSP_EOVERFLOW, "more than 2^20 matched keys");

  if (nmatch > 0) {
    // ---- S6: recovery and exact verification ----
    RecoverDev rd{};
    rd.match_key = pd.match_key;
    rd.match_cls = pd.match_cls;
    rd.nmatch = nmatch;
    rd.side[0] = pd.side[0];
    rd.side[1] = pd.side[1];
    rd.oidx[0] = bd[0].idx;
    rd.iidx[0] = bd[1].idx;
    rd.oidx[1] = bd[2].idx;
    rd.iidx[1] = bd[3].idx;
    rd.cmask = cmask;
    unsigned long long *tmp64;
    CK(da.get(&tmp64, (nmatch + 1 + 4095) / 4096 + 1));
    for (int side = 0; side < 2; ++side) {
      CK(da.get(&rd.cand_count[side], nmatch));
      CK(da.get(&rd.cand_off[side], nmatch + 1));
      CK(da.get(&rd.cand_cur[side], nmatch));
      CK(cudaMemsetAsync(rd.cand_count[side], 0, sizeof(unsigned long long) * nmatch, s));
      CK(cudaMemsetAsync(rd.cand_cur[side], 0, sizeof(unsigned long long) * nmatch, s));
    }
    CK(launch_recover(rd, false, s));
    unsigned long long ncand[2];
    for (int side = 0; side < 2; ++side) {
      CK(launch_scan_u64(rd.cand_count[side], rd.cand_off[side], nmatch, tmp64, s));
      CK(cudaMemcpyAsync(&ncand[side], rd.cand_off[side] + nmatch, sizeof(unsigned long long),
                         cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    for (int side = 0; side < 2; ++side) {
      rd.cand_cap[side] = ncand[side];
      CK(da.get(&rd.cand[side], ncand[side]));
    }
    CK(da.get(&rd.cand_match[0], ncand[0]));
    CK(launch_recover(rd, true, s));

    VerifyDev vd{};
    vd.ic = ic;
    for (int k = 0; k < 4; ++k) {
      vd.qvec[k] = qd[k].vec;
      vd.qsize[k] = qd[k].size;
    }
    vd.candL = rd.cand[0];
    vd.candL_match = rd.cand_match[0];
    vd.nL = ncand[0];
    vd.candR = rd.cand[1];
    vd.candR_off = rd.cand_off[1];
    unsigned long long *cnts;
    CK(da.get(&cnts, 2));
    vd.sol_count = cnts;
    vd.pairs_checked = cnts + 1;
    uint64_t cap = 1u << 16;
    for (int attempt = 0; attempt < 2; ++attempt) {
      CK(da.get(&vd.sol, 2 * cap));
      vd.sol_cap = cap;
      CK(cudaMemsetAsync(cnts, 0, 2 * sizeof(unsigned long long), s));
      CK(launch_verify(vd, s));
      unsigned long long hc[2];
      CK(cudaMemcpyAsync(hc, cnts, sizeof(hc), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      st.pairs_verified = hc[1];
      if (hc[0] <= cap) {
        res->masks.resize(2 * hc[0]);
        if (hc[0]) {
          CK(cudaMemcpyAsync(res->masks.data(), vd.sol, sizeof(uint64_t) * 2 * hc[0], cudaMemcpyDeviceToHost, s));
          CK(cudaStreamSynchronize(s));
        }
        break;
      }
      if (hc[0] > (1ull << 28)) return fail(MSP_EOVERFLOW, "more than 2^28 solutions");
      cap = hc[0];
    }
  }
  st.device_bytes = da.peak;
  da.release();
  CK(cudaStreamSynchronize(s));
  return MSP_OK;
}

int finish_solutions(const std::vector<uint64_t> &raw, int n, uint64_t **masks, size_t *count,
                            int *words) {
  const int W = (n + 63) / 64;
  const size_t cnt = raw.size() / 2;
  std::vector<std::pair<uint64_t, uint64_t>> v(cnt);
  for (size_t i = 0; i < cnt; ++i) v[i] = {raw[2 * i + 1], raw[2 * i]};  // (hi, lo)
  std::sort(v.begin(), v.end());
  v.erase(std::unique(v.begin(), v.end()), v.end());
  *count = v.size();
  if (words) *words = W;
  *masks = nullptr;
  if (v.empty()) return MSP_OK;
  auto *buf = static_cast<uint64_t *>(std::malloc(sizeof(uint64_t) * W * v.size()));
  if (!buf) return fail(MSP_ENOMEM, "host allocation of the solution list failed");
  for (size_t i = 0; i < v.size(); ++i) {
    buf[W * i] = v[i].second;
    if (W > 1) buf[W * i + 1] = v[i].first;
  }
  *masks = buf;
  return MSP_OK;
}

}  // namespace

namespace msp {

int solve_instance(msp_instance *inst, uint64_t **masks, size_t *count, int *words_per_mask) {
  if (!inst || !masks || !count) return fail(MSP_EINVAL, "null argument");
  *masks = nullptr;
  *count = 0;
  if (words_per_mask) *words_per_mask = (inst->n + 63) / 64;
  if (cudaSetDevice(inst->device) != cudaSuccess) return fail(MSP_ECUDA, "cudaSetDevice failed");
  const auto t0 = std::chrono::steady_clock::now();
  SolveResult res;
  int rc = solve_impl(inst, &res);
  if (rc != MSP_OK) {
    cudaStreamSynchronize(inst->stream);
    cudaGetLastError();
    return rc;
  }
  rc = finish_solutions(res.masks, inst->n, masks, count, words_per_mask);
  inst->stats.solutions = *count;
  inst->stats.ms_total =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return rc;
}

// Device bytes a solve of an (m, n) instance needs for its quarter lists and
// one residue pass of at least one class, capped at `cap` (0 = no cap).
size_t footprint_estimate(int m, int n, size_t cap) {
  const Plan p = make_plan(m, n);
  double fixed = 0;
  for (int k = 0; k < 4; ++k) fixed += std::ldexp(1.0, p.q[k]) * (8.0 * p.W + 16.0 + 16.0);
  fixed += 4.0 * std::ldexp(1.0, p.B) * 4.0 + (64 << 20);
  const double cls = (std::ldexp(1.0, p.lgL - p.B) + std::ldexp(1.0, p.lgR - p.B)) * 8.0 * 1.08;
  const double all = cls * std::ldexp(1.0, p.B);
  double want = fixed + std::min(all, std::max(cls, 4.0 * (1 << 30)));
  if (cap && want > (double)cap) want = std::max<double>(cap, fixed + cls);
  return static_cast<size_t>(want);
}

}  // namespace msp

extern "C" {

const char *msp_last_error(void) { return g_err.c_str(); }

const char *msp_version(void) { return "libmsp 0.1 (sm_103a)"; }

int msp_create(const int32_t *A, const int32_t *d, int m, int n, msp_instance **out) {
  if (!out) return fail(MSP_EINVAL, "out must be non-null");
  *out = nullptr;
  int rc = validate(A, d, m, n);
  if (rc != MSP_OK) return rc;
  int dev_count = 0;
  cudaError_t e = cudaGetDeviceCount(&dev_count);
  if (e != cudaSuccess || dev_count < 1) return fail(MSP_ECUDA, "no CUDA device available");
  auto *inst = new (std::nothrow) msp_instance();
  if (!inst) return fail(MSP_ENOMEM, "host allocation failed");
  inst->m = m;
  inst->n = n;
  inst->A.assign(A, A + (size_t)m * n);
  inst->d.assign(d, d + m);
  cudaGetDevice(&inst->device);
  {
    // keep freed pass buffers in the stream-ordered pool between solves
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, inst->device) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  }
  e = cudaStreamCreateWithFlags(&inst->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete inst;
    return fail(MSP_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
  }
  inst->own_stream = true;
  *out = inst;
  return MSP_OK;
}

void msp_destroy(msp_instance *inst) {
  if (!inst) return;
  if (inst->stream) cudaStreamSynchronize(inst->stream);
  if (inst->own_stream && inst->stream) cudaStreamDestroy(inst->stream);
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, inst->device) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
  delete inst;
}

int msp_set_stream(msp_instance *inst, void *cuda_stream) {
  if (!inst) return fail(MSP_EINVAL, "null instance");
  if (inst->own_stream && inst->stream) cudaStreamDestroy(inst->stream);
  inst->own_stream = false;
  inst->stream = static_cast<cudaStream_t>(cuda_stream);
  if (!cuda_stream) {
    if (cudaStreamCreateWithFlags(&inst->stream, cudaStreamNonBlocking) != cudaSuccess)
      return fail(MSP_ECUDA, "cudaStreamCreate failed");
    inst->own_stream = true;
  }
  return MSP_OK;
}

int msp_set_memory_budget(msp_instance *inst, size_t bytes) {
  if (!inst) return fail(MSP_EINVAL, "null instance");
  inst->budget = bytes;
  return MSP_OK;
}

int msp_solve_all(msp_instance *inst, uint64_t **masks, size_t *count, int *words_per_mask) {
  return msp::solve_instance(inst, masks, count, words_per_mask);
}

int msp_get_stats(const msp_instance *inst, msp_stats *out) {
  if (!inst || !out) return fail(MSP_EINVAL, "null argument");
  *out = inst->stats;
  return MSP_OK;
}

void msp_free_solutions(uint64_t *masks) { std::free(masks); }

int msp_solve_batch(const int32_t *const *A, const int32_t *const *d, int m, int n, int count,
                    uint64_t **masks, size_t *offsets) {
  if (!A || !d || !masks || !offsets || count < 0) return fail(MSP_EINVAL, "null argument");
  *masks = nullptr;
  const int W = (n + 63) / 64;
  std::vector<uint64_t> all;
  offsets[0] = 0;
  for (int k = 0; k < count; ++k) {
    msp_instance *inst = nullptr;
    int rc = msp_create(A[k], d[k], m, n, &inst);
    if (rc != MSP_OK) return rc;
    uint64_t *mk = nullptr;
    size_t c = 0;
    rc = msp_solve_all(inst, &mk, &c, nullptr);
    msp_destroy(inst);
    if (rc != MSP_OK) return rc;
    all.insert(all.end(), mk, mk + c * W);
    msp_free_solutions(mk);
    offsets[k + 1] = offsets[k] + c;
  }
  if (!all.empty()) {
    *masks = static_cast<uint64_t *>(std::malloc(sizeof(uint64_t) * all.size()));
    if (!*masks) return fail(MSP_ENOMEM, "host allocation failed");
    std::memcpy(*masks, all.data(), sizeof(uint64_t) * all.size());
  }
  return MSP_OK;
}

}  // extern "C"
