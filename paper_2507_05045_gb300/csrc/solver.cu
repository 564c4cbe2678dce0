// Host side of libmsp: validation, the pass planner and the C ABI of
// include/msp.h.  Every arithmetic step of a solve runs in the kernels of
// kernels.cu; the host only plans, allocates, launches and collects.
#include "msp_internal.cuh"
#include "../../include/msp.h"
#include "host_internal.h"
#include "host_util.h"

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

// Quarters: sizes ceil(n/4) for the first n mod 4 quarters, floor(n/4) for
// the rest; L pairs the largest quarter Q1 with Q3, R pairs Q2 with Q4.
Plan make_plan(int m, int n, const PlanChoice &ch) {
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
  // about 2^21 records per class and side (at most 2^23 classes).  Halves
  // of 44 to 47 columns keep classes of 2^21 records with inner buckets of
  // about 32 elements (inner quarters of B + 5 columns), so a scatter window
  // expands half as many outer elements per round (measured on the (10,90)
  // class: 3.4 % faster passes than 2^25 classes of 2^20 records with
  // buckets of 16).  Halves of 48 columns or more take classes of about
  // 2^20 records, up to 2^27 of them: fewer digits per class (measured on
  // the (11,100) class: 23 % faster than 2^26 classes).
  p.B = ch.B >= 0 ? std::min(kMaxStreamClassBits, ch.B) : std::min(23, std::max(0, lgmax - 21));
  if (ch.B < 0 && lgmax >= 44) p.B = std::min(kMaxStreamClassBits, lgmax >= 48 ? lgmax - 20 : lgmax - 21);
  // row 1 alone while its residues stay uniform (2^B <= 256 against a
  // row-1 spread of a few hundred); three rows beyond, which keeps the class
  // sizes within about one percent of each other (four rows past 2^18
  // classes)
  p.t = p.B <= 8 ? 1 : (p.B <= 18 ? 3 : 4);
  p.t = std::min(p.t, m);
  // Uneven halves: the inner quarter of each side (Q3 of L, Q4 of R) takes
  // columns from the outer one until an inner residue bucket holds about 16
  // elements (2^(q_inner - B); 32 for halves of 44 to 47 columns), at most
  // 2^27 of them (2^30 for the plans of more than 2^23 classes or halves of
  // 44 columns or more, whose lists then take up to about 120 GB), so that
  // every outer element of a scatter window expands to a run of consecutive
  // inner keys.  |L| and |R| do not change, nor do the classes and
  // partitions.
  const int inner_bits = ch.inner >= 0 ? ch.inner : (lgmax >= 44 && lgmax < 48 ? 5 : 4);
  const int inner_cap = p.B > 23 || lgmax >= 44 ? 30 : 27;
  for (int side = 0; side < 2; ++side) {
    const int tot = p.q[side] + p.q[side + 2];
    const int want = std::min({std::max(p.q[side + 2], p.B + inner_bits), inner_cap, tot - 1});
    if (want > p.q[side + 2]) {
      p.q[side + 2] = want;
      p.q[side] = tot - want;
    }
  }
  c = 0;
  for (int k = 0; k < 4; ++k) {
    p.col0[k] = c;
    c += p.q[k];
  }
  // partitions of about 2^12 records (512 digits for a class of 2^21),
  // in the streaming and in the exact two-phase pass
  p.D = ch.D >= 0 ? std::min(12, ch.D) : std::min(12, std::max(0, lgmax - p.B - 12));
  p.Dx = std::min(12, std::max(0, lgmax - p.B - 12));
  p.S = 11;  // 2048 shared-memory buckets per partition side
  uint64_t s = 0x2507050450000001ull;
  p.c_row[0] = 1;
  for (int i = 1; i < kMaxClassRows; ++i) p.c_row[i] = static_cast<uint32_t>(splitmix(s)) | 1u;
  for (int i = 0; i < kMaxRows; ++i) p.w_row[i] = splitmix(s) | 1ull;
  return p;
}

}  // namespace msp

using namespace msp;

namespace {

}  // namespace

namespace msp {
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

size_t solve_budget(const msp_instance *inst, size_t already_held) {
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return inst->budget;
  }
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, inst->device) == cudaSuccess) {
    uint64_t reserved = 0, used = 0;
    cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved);
    cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used);
    if (reserved > used) free_b += reserved - used;
  }
  const double avail = (double)free_b + (double)already_held;
  size_t budget = inst->budget ? inst->budget : static_cast<size_t>(0.85 * avail);
  return std::min(budget, static_cast<size_t>(0.95 * avail));
}
}  // namespace msp

namespace {

struct SolveResult {
  std::vector<uint64_t> masks;  // [count][2]
};

// The solve proper.  `out` receives unsorted solution masks (two words each).
int solve_impl(msp_instance *inst, SolveResult *res) {
  const int m = inst->m, n = inst->n;
  PlanChoice ch;
  ch.B = inst->plan_B;
  ch.D = inst->plan_D;
  ch.inner = inst->plan_inner;
  const Plan p = make_plan(m, n, ch);
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

  // ---- the direct pass (direct.cu) for every instance it fits ----
  {
    const bool stream_plan = inst->plan_B >= 0 || inst->plan_D >= 0 || inst->plan_inner >= 0;
    const bool want = !inst->force_exact && (inst->direct == 1 || (inst->direct < 0 && !stream_plan));
    const DirectPlan dp = make_direct_plan(m, n, inst->table_bits);
    if (want && dp.ok) {
      const msp_stats st0 = st;
      Prof dprof;
      dprof.on = inst->profiling;
      dprof.s = s;
      dprof.st = &st;
      std::vector<uint64_t> raw;
      const int rc = solve_direct(inst, dp, p, solve_budget(inst, 0), dprof, raw);
      if (rc == MSP_OK) {
        st.path = 1;
        res->masks = std::move(raw);
        return MSP_OK;
      }
      if (rc != kDirectFallback) return rc;
      // the streaming and exact passes solve it; the direct attempt's
      // launches stay counted
      const uint64_t launches = st.kernel_launches;
      st = st0;
      st.kernel_launches = launches;
      st.direct_fallback = 1;
    }
  }

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

  Prof prof;
  prof.on = inst->profiling;
  prof.s = s;
  prof.st = &st;
  auto h2d = [&](void *dst, const void *hsrc, size_t b) {
    st.h2d_bytes += b;
    return cudaMemcpyAsync(dst, hsrc, b, cudaMemcpyHostToDevice, s);
  };
  auto d2h = [&](void *hdst, const void *dsrc, size_t b) {
    st.d2h_bytes += b;
    return cudaMemcpyAsync(hdst, dsrc, b, cudaMemcpyDeviceToHost, s);
  };
  DevAlloc da(s);
  uint64_t *d_pcol, *d_kcol;
  uint32_t *d_ccol;
  CK(da.get(&d_pcol, pcol.size()));
  CK(da.get(&d_kcol, kcol.size()));
  CK(da.get(&d_ccol, ccol.size()));
  CK(h2d(d_pcol, pcol.data(), pcol.size() * 8));
  CK(h2d(d_kcol, kcol.data(), kcol.size() * 8));
  CK(h2d(d_ccol, ccol.data(), ccol.size() * 4));

  // ---- S1: quarter lists ----
  NvtxRange nv_lists("msp: quarter lists and class buckets");
  QuarterDev qd[4];
  for (int k = 0; k < 4; ++k) {
    qd[k].q = p.q[k];
    qd[k].size = int64_t(1) << p.q[k];
    CK(da.get(&qd[k].vec, (size_t)p.W * qd[k].size));
    CK(da.get(&qd[k].key, qd[k].size));
    CK(da.get(&qd[k].cls, qd[k].size));
    CK(da.get(&qd[k].v1, qd[k].size));
    LAUNCH(MSP_K_GRAY, 1, 0, launch_gray(ic, d_pcol, d_kcol, d_ccol, qd[k], p.col0[k], s));
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
    LAUNCH(MSP_K_BUCKET, 1, 0, launch_count_classes(q.cls, q.size, static_cast<uint32_t>(mul[l]), cadd[l], cmask, d_hist, s));
    LAUNCH(MSP_K_BUCKET, 3, 0, launch_scan_u32(d_hist, bd[l].off, M, d_scantmp, s));
    CK(cudaMemcpyAsync(d_cursor, bd[l].off, sizeof(uint32_t) * M, cudaMemcpyDeviceToDevice, s));
    LAUNCH(MSP_K_BUCKET, 1, 0, launch_bucket_scatter(q, mul[l], kadd[l], cadd[l], cmask, d_cursor, bd[l], s));
  }

  nv_lists.end();
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
      LAUNCH(MSP_K_C1, 1, 0, launch_v1_hist(qd[k].v1, qd[k].size, h[k], s));
    }
    CK(da.get(&hl, lenl));
    CK(da.get(&hr, lenr));
    CK(da.get(&c1, 2));
    LAUNCH(MSP_K_C1, 3, 0, launch_row1_candidates(h[0], h[2], len13, h[1], h[3], len24, hl, hr, lenl, lenr, inst->d[0], c1, s));
    unsigned long long c1h[2];
    CK(d2h(c1h, c1, sizeof(c1h)));
    CK(cudaStreamSynchronize(s));
    st.row1_candidates_lo = c1h[0];
    st.row1_candidates_hi = c1h[1];
  }

  // ---- pass setup ----
  const int nd = 1 << p.D;
  SideGen gens[2];
  for (int side = 0; side < 2; ++side) {
    const BucketDev &o = bd[side == 0 ? 0 : 2];
    const BucketDev &in = bd[side == 0 ? 1 : 3];
    SideGen &g = gens[side];
    g.okey = o.key;
    g.ocls = o.cls;
    g.osize = o.size;
    g.ikey = in.key;
    g.isize = in.size;
    g.ioff = in.off;
    const int64_t per_bucket = std::max<int64_t>(1, in.size / M);
    g.slice_outer = std::max<int64_t>(1, (int64_t(1) << 19) / per_bucket);
    g.slices = static_cast<int>((o.size + g.slice_outer - 1) / g.slice_outer);
    g.wmax = scatter_window(in.size, M);
  }
  // memory budget: free device memory, plus what the stream-ordered pool
  // holds unused from earlier solves, plus this solve's own allocations
  const size_t budget = solve_budget(inst, da.bytes);
  const size_t fixed_reserve = (size_t)64 << 20;  // matches and small per-pass tables

  uint64_t *match_key;
  uint32_t *match_cls;
  unsigned long long *match_count;
  const uint64_t match_cap = 1u << 20;
  CK(da.get(&match_key, match_cap));
  CK(da.get(&match_cls, match_cap));
  CK(da.get(&match_count, 1));
  CK(cudaMemsetAsync(match_count, 0, sizeof(unsigned long long), s));

  // ---- S6: recovery and exact verification of the matches [m0, m1);
  //      solutions are appended to res (two words each) ----
  uint64_t verified_to = 0;
  auto verify_matches = [&](uint64_t m0, uint64_t m1) -> int {
    const uint64_t nm = m1 - m0;
    RecoverDev rd{};
    rd.match_key = match_key + m0;
    rd.match_cls = match_cls + m0;
    rd.nmatch = nm;
    rd.side[0] = gens[0];
    rd.side[1] = gens[1];
    rd.oidx[0] = bd[0].idx;
    rd.iidx[0] = bd[1].idx;
    rd.oidx[1] = bd[2].idx;
    rd.iidx[1] = bd[3].idx;
    rd.cmask = cmask;
    unsigned long long *tmp64;
    CK(da.get(&tmp64, (nm + 1 + 4095) / 4096 + 1));
    for (int side = 0; side < 2; ++side) {
      CK(da.get(&rd.cand_count[side], nm));
      CK(da.get(&rd.cand_off[side], nm + 1));
      CK(da.get(&rd.cand_cur[side], nm));
      CK(cudaMemsetAsync(rd.cand_count[side], 0, sizeof(unsigned long long) * nm, s));
      CK(cudaMemsetAsync(rd.cand_cur[side], 0, sizeof(unsigned long long) * nm, s));
    }
    LAUNCH(MSP_K_RECOVER, 2, 0, launch_recover(rd, false, s));
    unsigned long long ncand[2];
    for (int side = 0; side < 2; ++side) {
      LAUNCH(MSP_K_RECOVER, 3, 0, launch_scan_u64(rd.cand_count[side], rd.cand_off[side], nm, tmp64, s));
      CK(d2h(&ncand[side], rd.cand_off[side] + nm, sizeof(unsigned long long)));
    }
    CK(cudaStreamSynchronize(s));
    for (int side = 0; side < 2; ++side) {
      rd.cand_cap[side] = ncand[side];
      CK(da.get(&rd.cand[side], ncand[side]));
    }
    CK(da.get(&rd.cand_match[0], ncand[0]));
    LAUNCH(MSP_K_RECOVER, 2, 0, launch_recover(rd, true, s));

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
      LAUNCH(MSP_K_VERIFY, vd.nL ? 1 : 0, 0, launch_verify(vd, s));
      unsigned long long hc[2];
      CK(d2h(hc, cnts, sizeof(hc)));
      CK(cudaStreamSynchronize(s));
      if (hc[0] <= cap) {
        st.pairs_verified += hc[1];
        const size_t at = res->masks.size();
        res->masks.resize(at + 2 * hc[0]);
        if (hc[0]) {
          CK(d2h(res->masks.data() + at, vd.sol, sizeof(uint64_t) * 2 * hc[0]));
          CK(cudaStreamSynchronize(s));
        }
        return MSP_OK;
      }
      if (hc[0] > (1ull << 28)) return fail(MSP_EOVERFLOW, "more than 2^28 solutions");
      cap = hc[0];
    }
    return MSP_OK;
  };

  uint64_t *rec[2] = {nullptr, nullptr};
  uint64_t rec_cap[2] = {0, 0};
  // (re)allocate the record buffers to hold at least need[] records
  auto ensure_rec = [&](const uint64_t need[2]) -> cudaError_t {
    for (int side = 0; side < 2; ++side) {
      if (need[side] <= rec_cap[side]) continue;
      if (rec[side]) da.free1(rec[side], sizeof(uint64_t) * rec_cap[side]);
      rec[side] = nullptr;
      rec_cap[side] = 0;
      cudaError_t e = da.get(&rec[side], need[side]);
      if (e != cudaSuccess) return e;
      rec_cap[side] = need[side];
    }
    return cudaSuccess;
  };

  if (inst->part >= inst->parts) return fail(MSP_EINVAL, "class part must be below the number of parts");
  const uint32_t c_begin = static_cast<uint32_t>((uint64_t)M * inst->part / inst->parts);
  const uint32_t c_end = static_cast<uint32_t>((uint64_t)M * (inst->part + 1) / inst->parts);
  st.classes_total = M;
  st.classes_done = c_end - c_begin;
  int passes = 0;
  uint64_t oversize = 0;
  bool found_first = false;  // time to first: a pass yielded a solution, the rest is skipped
  std::vector<std::pair<uint32_t, uint32_t>> exact_ranges;
  bool fast = !inst->force_exact && c_begin < c_end;
  std::vector<unsigned long long> csz[2];
  std::vector<uint32_t> capv[2];
  if (fast) {
    // exact sizes of the classes to enumerate, by convolution of the bucket
    // histograms (S2); O(M) work per class
    const uint32_t ncl = c_end - c_begin;
    unsigned long long *d_csz;
    CK(da.get(&d_csz, 2 * (size_t)ncl));
    // the cheaper form: over the M outer buckets, or over the outer elements
    // when they are fewer (many classes, e.g. the n = 100 plans)
    for (int side = 0; side < 2; ++side) {
      const BucketDev &o = bd[side == 0 ? 0 : 2];
      const BucketDev &in = bd[side == 0 ? 1 : 3];
      if (o.size < (int64_t)M) {
        LAUNCH(MSP_K_OTHER, 1, 0,
               launch_class_sizes_elems(o.cls, o.size, in.off, M, c_begin, ncl, d_csz + (size_t)side * ncl, s));
      } else {
        LAUNCH(MSP_K_OTHER, 1, 0, launch_class_sizes(o.off, in.off, M, c_begin, ncl, d_csz + (size_t)side * ncl, s));
      }
    }
    for (int side = 0; side < 2; ++side) {
      csz[side].assign(M, 0);
      capv[side].assign(M, 0);
      CK(d2h(csz[side].data() + c_begin, d_csz + (size_t)side * ncl, sizeof(unsigned long long) * ncl));
    }
    CK(cudaStreamSynchronize(s));
    prof.flush();
    da.free1(d_csz, sizeof(unsigned long long) * 2 * ncl);
    // partition capacity mean + 7 sigma + 32 (a multiple of 16 records,
    // at most kFastCap); a class whose partitions would not hold even
    // mean + 4 sigma takes the exact path
    for (int side = 0; side < 2; ++side)
      for (uint32_t c = c_begin; c < c_end; ++c) {
        const double mean = (double)csz[side][c] / nd;
        uint64_t cap = static_cast<uint64_t>(std::ceil(mean + 7.0 * std::sqrt(mean) + 32.0));
        cap = std::min<uint64_t>((cap + 15) & ~uint64_t(15), kFastCap);
        const bool fits = mean + 4.0 * std::sqrt(mean) <= (double)kFastCap;
        capv[side][c] = fits ? static_cast<uint32_t>(cap) : 0u;
      }
  }
  if (fast) {
    // ---- streaming passes: greedy runs of classes whose partition regions
    //      fit the record budget ----
    const double rec_budget = std::max(0.0, (double)budget - (double)da.bytes - (double)fixed_reserve);
    double tot_region[2] = {0, 0};
    for (int side = 0; side < 2; ++side)
      for (uint32_t c = c_begin; c < c_end; ++c) tot_region[side] += (double)capv[side][c] * nd;
    const double frac0 = tot_region[0] / std::max(1.0, tot_region[0] + tot_region[1]);
    const uint64_t lim[2] = {static_cast<uint64_t>(rec_budget / 8.0 * frac0),
                             static_cast<uint64_t>(rec_budget / 8.0 * (1.0 - frac0))};
    const int max_run = 1 << 16;
    struct PassPlan {
      uint32_t c0, c1;
      uint64_t recs;
    };
    std::vector<PassPlan> plan;
    std::vector<uint64_t> base_h[2] = {std::vector<uint64_t>(M), std::vector<uint64_t>(M)};
    uint64_t need[2] = {0, 0};
    for (uint32_t c = c_begin; c < c_end; ++c) st.records_done += csz[0][c] + csz[1][c];
    for (uint32_t c0 = c_begin; c0 < c_end;) {
      if (capv[0][c0] == 0 || capv[1][c0] == 0) {  // oversized class: exact path
        if (!exact_ranges.empty() && exact_ranges.back().second == c0)
          exact_ranges.back().second = c0 + 1;
        else
          exact_ranges.push_back({c0, c0 + 1});
        ++c0;
        continue;
      }
      uint64_t acc[2] = {0, 0}, recs = 0;
      uint32_t c = c0;
      while (c < c_end && (int)(c - c0) < max_run && capv[0][c] && capv[1][c]) {
        const uint64_t r0 = (uint64_t)capv[0][c] * nd, r1 = (uint64_t)capv[1][c] * nd;
        if (c > c0 && (acc[0] + r0 > lim[0] || acc[1] + r1 > lim[1])) break;
        base_h[0][c] = acc[0];
        base_h[1][c] = acc[1];
        acc[0] += r0;
        acc[1] += r1;
        recs += csz[0][c] + csz[1][c];
        ++c;
      }
      plan.push_back({c0, c, recs});
      need[0] = std::max(need[0], acc[0]);
      need[1] = std::max(need[1], acc[1]);
      c0 = c;
    }
    if ((double)(need[0] + need[1]) * 8.0 > (double)budget - (double)da.bytes)
      return fail(MSP_ENOMEM, "memory budget too small for one residue class");
    CK(ensure_rec(need));
    int max_c = 0;
    for (auto &pp : plan) max_c = std::max<int>(max_c, pp.c1 - pp.c0);
    uint64_t *d_base[2];
    uint32_t *d_cap[2], *d_fill[2];
    unsigned int *d_ovf, *d_err;
    for (int side = 0; side < 2; ++side) {
      CK(da.get(&d_base[side], M));
      CK(da.get(&d_cap[side], M));
      CK(da.get(&d_fill[side], (size_t)max_c * nd));
      CK(h2d(d_base[side], base_h[side].data(), sizeof(uint64_t) * M));
      CK(h2d(d_cap[side], capv[side].data(), sizeof(uint32_t) * M));
    }
    CK(da.get(&d_ovf, plan.size()));
    CK(da.get(&d_err, 1));
    CK(cudaMemsetAsync(d_ovf, 0, sizeof(unsigned int) * plan.size(), s));
    CK(cudaMemsetAsync(d_err, 0, sizeof(unsigned int), s));
    FastInst fi{};
    for (int side = 0; side < 2; ++side) {
      fi.side[side] = gens[side];
      fi.class_base[side] = d_base[side];
      fi.cap[side] = d_cap[side];
      fi.fill[side] = d_fill[side];
    }
    fi.tag = 0;
    FastInst *d_fi;
    CK(da.get(&d_fi, 1));
    CK(h2d(d_fi, &fi, sizeof(FastInst)));
    FastPass fp{};
    fp.inst = d_fi;
    fp.ninst = 1;
    fp.slices[0] = gens[0].slices;
    fp.slices[1] = gens[1].slices;
    fp.cmask = cmask;
    fp.D = p.D;
    fp.S = p.S;
    fp.rec[0] = rec[0];
    fp.rec[1] = rec[1];
    fp.error = d_err;
    fp.wait_ns = inst->wait_ns;
    fp.wait_check = inst->wait_check;
    fp.match_key = match_key;
    fp.match_cls = match_cls;
    fp.match_count = match_count;
    fp.match_cap = match_cap;
    uint64_t recs_run = 0;
    uint32_t classes_run = 0;
    size_t passes_run = 0;
    for (size_t k = 0; k < plan.size(); ++k) {
      if (inst->cancel && *inst->cancel) return fail(MSP_ECANCELED, "request canceled");
      const PassPlan &pp = plan[k];
      const int run = static_cast<int>(pp.c1 - pp.c0);
      fp.c0 = static_cast<int>(pp.c0);
      fp.nclass = run;
      for (int side = 0; side < 2; ++side)
        CK(cudaMemsetAsync(d_fill[side], 0, sizeof(uint32_t) * (size_t)run * nd, s));
      fp.overflow = d_ovf + k;
      LAUNCH(MSP_K_GEN_SCATTER, 1, 8 * pp.recs, launch_scatter_fast(fp, run, s));
      LAUNCH(MSP_K_JOIN, 1, 8 * pp.recs, launch_join_fast(fp, run, s));
      ++passes;
      ++passes_run;
      recs_run += pp.recs;
      classes_run += static_cast<uint32_t>(run);
      if (inst->first_only) {
        // time to first: verify this pass's new matches and stop at the
        // first pass that yields a solution (a pass whose partitions
        // overflowed may have missed matches; it is re-run exactly below
        // unless a solution turns up first)
        unsigned int err1 = 0;
        unsigned long long nm = 0;
        CK(d2h(&err1, d_err, sizeof(err1)));
        CK(d2h(&nm, match_count, sizeof(nm)));
        CK(cudaStreamSynchronize(s));
        prof.flush();
        if (err1) return fail(MSP_ETIMEDOUT, "a bulk copy did not complete within its time limit");
        if (nm > match_cap) return fail(MSP_EOVERFLOW, "more than 2^20 matched keys");
        if (nm > verified_to) {
          const int rc = verify_matches(verified_to, nm);
          if (rc != MSP_OK) return rc;
          verified_to = nm;
        }
        if (!res->masks.empty()) {
          found_first = true;
          break;
        }
      }
    }
    if (found_first) {
      st.classes_done = classes_run;
      st.records_done = recs_run;
    }
    std::vector<unsigned int> ovf_h(plan.size());
    unsigned int err_h = 0;
    CK(d2h(ovf_h.data(), d_ovf, sizeof(unsigned int) * plan.size()));
    CK(d2h(&err_h, d_err, sizeof(unsigned int)));
    CK(cudaStreamSynchronize(s));
    prof.flush();
    if (err_h) return fail(MSP_ETIMEDOUT, "a bulk copy did not complete within its time limit");
    for (size_t k = 0; k < passes_run && !found_first; ++k)
      if (ovf_h[k]) {
        exact_ranges.push_back({plan[k].c0, plan[k].c1});
        ++st.fast_passes_redone;
      }
  } else if (c_begin < c_end) {
    exact_ranges.push_back({c_begin, c_end});
  }

  if (!exact_ranges.empty() && !found_first) {
    const int nd = 1 << p.Dx;  // exact pass digits
    // ---- exact passes: count, offsets, scatter, shared-memory join; any
    //      partition larger than shared memory goes to join_big ----
    PassDev pd{};
    pd.cmask = cmask;
    pd.D = p.Dx;
    pd.S = p.S;
    pd.side[0] = gens[0];
    pd.side[1] = gens[1];
    const double est_class[2] = {std::ldexp(1.0, p.lgL - p.B), std::ldexp(1.0, p.lgR - p.B)};
    const size_t per_class_meta =
        (size_t)nd * (sizeof(uint64_t) + sizeof(uint32_t)) * 2 +
        (size_t)nd * sizeof(uint32_t) * (pd.side[0].slices + pd.side[1].slices) + 64;
    const double per_class_bytes = (est_class[0] + est_class[1]) * 8.0 * 1.08 + per_class_meta;
    const double room = (double)budget - (double)da.bytes + 8.0 * (double)(rec_cap[0] + rec_cap[1]);
    if (room < fixed_reserve + per_class_bytes)
      return fail(MSP_ENOMEM, "memory budget too small for one residue class");
    int max_classes = static_cast<int>(std::min<double>(M, std::floor((room - fixed_reserve) / per_class_bytes)));
    max_classes = std::max(1, std::min(max_classes, 1 << 16));
    {
      const uint64_t need[2] = {
          static_cast<uint64_t>(std::min<double>(std::ldexp(1.0, p.lgL), est_class[0] * 1.08 * max_classes + 4096)),
          static_cast<uint64_t>(std::min<double>(std::ldexp(1.0, p.lgR), est_class[1] * 1.08 * max_classes + 4096))};
      CK(ensure_rec(need));
    }
    for (int side = 0; side < 2; ++side) {
      CK(da.get(&pd.cnt[side], (size_t)max_classes * pd.side[side].slices * nd));
      CK(da.get(&pd.segstart[side], (size_t)max_classes * nd));
      CK(da.get(&pd.seglen[side], (size_t)max_classes * nd));
      CK(da.get(&pd.classtot[side], (size_t)max_classes));
      CK(da.get(&pd.classbase[side], (size_t)max_classes));
    }
    pd.match_key = match_key;
    pd.match_cls = match_cls;
    pd.match_count = match_count;
    pd.match_cap = match_cap;
    pd.big_cap = static_cast<uint32_t>(std::min<uint64_t>((uint64_t)max_classes * nd, 1u << 24));
    CK(da.get(&pd.big_list, pd.big_cap));
    CK(da.get(&pd.big_count, 1));

    std::vector<uint64_t> tot_h(2 * (size_t)max_classes), base_h(2 * (size_t)max_classes);
    unsigned int big_h = 0;
    for (const auto &range : exact_ranges) {
      for (uint32_t c0 = range.first; c0 < range.second;) {
        if (inst->cancel && *inst->cancel) return fail(MSP_ECANCELED, "request canceled");
        pd.rec[0] = rec[0];
        pd.rec[1] = rec[1];
        pd.c0 = static_cast<int>(c0);
        pd.nclass = static_cast<int>(std::min<uint64_t>(max_classes, range.second - c0));
        LAUNCH(MSP_K_GEN_COUNT, 1, 0, launch_gen_count(pd, s));
        LAUNCH(MSP_K_OFFSETS, 1, 0, launch_counts_to_offsets(pd, s));
        CK(d2h(tot_h.data(), pd.classtot[0], sizeof(uint64_t) * pd.nclass));
        CK(d2h(tot_h.data() + max_classes, pd.classtot[1], sizeof(uint64_t) * pd.nclass));
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
        if (!fast) st.records_done += acc[0] + acc[1];
        if (run == 0) {
          // A class larger than the buffers (skewed class sizes): grow them
          // to hold it if the budget allows, then retry the pass.
          const uint64_t need[2] = {tot_h[0], tot_h[max_classes]};
          const double need_bytes = 8.0 * (double)(need[0] + need[1]) + (double)da.bytes -
                                    8.0 * (double)(rec_cap[0] + rec_cap[1]);
          if (need[0] >= (1ull << 31) || need[1] >= (1ull << 31) || need_bytes > (double)budget)
            return fail(MSP_ENOMEM, "one residue class does not fit the memory budget");
          CK(ensure_rec(need));
          continue;
        }
        CK(h2d(pd.classbase[0], base_h.data(), sizeof(uint64_t) * run));
        CK(h2d(pd.classbase[1], base_h.data() + max_classes, sizeof(uint64_t) * run));
        LAUNCH(MSP_K_GEN_SCATTER, 1, 8 * (acc[0] + acc[1]), launch_gen_scatter(pd, run, s));
        CK(cudaMemsetAsync(pd.big_count, 0, sizeof(unsigned int), s));
        LAUNCH(MSP_K_JOIN, 1, 8 * (acc[0] + acc[1]), launch_join(pd, run, s));
        LAUNCH(MSP_K_JOIN_BIG, 1, 0, launch_join_big(pd, run, s));
        CK(d2h(&big_h, pd.big_count, sizeof(unsigned int)));
        CK(cudaStreamSynchronize(s));
        prof.flush();
        oversize += big_h;
        if (big_h > pd.big_cap) return fail(MSP_EOVERFLOW, "too many oversize partitions in one pass");
        c0 += static_cast<uint32_t>(run);
        ++passes;
      }
    }
  }
  st.passes = passes;
  st.oversize_segments = oversize;

  unsigned long long nmatch = 0;
  CK(d2h(&nmatch, match_count, sizeof(nmatch)));
  CK(cudaStreamSynchronize(s));
  st.key_matches = nmatch;
  if (nmatch > match_cap) return fail(MSP_EOVERFLOW, "more than 2^20 matched keys");

  if (nmatch > verified_to && !found_first) {
    const int rc = verify_matches(verified_to, nmatch);
    if (rc != MSP_OK) return rc;
  }
  st.device_bytes = da.peak;
  da.release();
  CK(cudaStreamSynchronize(s));
  prof.flush();
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
  NvtxRange nv("msp_solve_all");
  if (cudaSetDevice(inst->device) != cudaSuccess) return fail(MSP_ECUDA, "cudaSetDevice failed");
  const auto t0 = std::chrono::steady_clock::now();
  SolveResult res;
  int rc = solve_impl(inst, &res);
  if (kChecked) {  // MSP_CHECKED build: any failed bounds check fails the solve
    const unsigned site = take_check_sites();
    if (site)
      return fail(MSP_ECUDA, "MSP_CHECKED: a bounds check failed at site " + std::to_string(site) +
                                 " (the access was skipped)");
  }
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
namespace {
std::vector<CheckReader> &check_readers() {
  static std::vector<CheckReader> r;
  return r;
}
}  // namespace

void register_check_reader(CheckReader r) { check_readers().push_back(r); }

unsigned take_check_sites() {
  if (!kChecked) return 0;
  cudaDeviceSynchronize();
  unsigned first = 0;
  for (CheckReader r : check_readers()) {
    const unsigned s = r();
    if (s && !first) first = s;
  }
  return first;
}

size_t footprint_estimate(int m, int n, size_t cap) {
  {
    // the direct pass, when the instance fits it and its lists fit the cap
    const DirectPlan dp = make_direct_plan(m, n, -1);
    if (dp.ok) {
      const size_t dneed = direct_footprint(dp);
      if (!cap || dneed <= cap) return dneed;
    }
  }
  const Plan p = make_plan(m, n);
  double fixed = 0;
  // quarter lists (packed rows, key, class, row 1) and their class buckets
  for (int k = 0; k < 4; ++k) fixed += std::ldexp(1.0, p.q[k]) * (8.0 * p.W + 16.0 + 16.0);
  // per-class tables (bucket offsets, class sizes, partition bases and caps)
  fixed += 64.0 * std::ldexp(1.0, p.B);
  // matched keys, the exact path's reserve, and a margin
  fixed += (12 << 20) + (64 << 20) + (64 << 20);
  const double cls = (std::ldexp(1.0, p.lgL - p.B) + std::ldexp(1.0, p.lgR - p.B)) * 8.0 * 1.1;
  const double all = cls * std::ldexp(1.0, p.B);
  double want = fixed + std::min(all, std::max(2.0 * cls, 4.0 * (1 << 30)));
  if (cap && want > (double)cap) want = std::max<double>(cap, fixed + 2.0 * cls);
  return static_cast<size_t>(want);
}

}  // namespace msp

extern "C" {

const char *msp_last_error(void) { return g_err.c_str(); }

const char *msp_version(void) {
  return msp::kChecked ? "libmsp 0.1 (sm_103a, MSP_CHECKED bounds checks)" : "libmsp 0.1 (sm_103a)";
}

int msp_plan(int m, int n, msp_plan_info *out) {
  if (!out) return fail(MSP_EINVAL, "out must be non-null");
  if (m < 1 || m > kMaxRows) return fail(MSP_ERANGE, "m must lie in [1, 16]");
  if (n < 1 || n > kMaxN) return fail(MSP_ERANGE, "n must lie in [1, 100]");
  std::memset(out, 0, sizeof(*out));
  const DirectPlan dp = make_direct_plan(m, n, -1);
  if (dp.ok) {
    out->path = 1;
    out->class_bits = dp.B;
    out->class_rows = dp.t;
    out->quarter[0] = dp.qo[0];
    out->quarter[1] = dp.qo[1];
    out->quarter[2] = dp.qi[0];
    out->quarter[3] = dp.qi[1];
    out->table_bits = dp.TB;
  } else {
    const Plan p = make_plan(m, n);
    out->path = 0;
    out->class_bits = p.B;
    out->class_rows = p.t;
    for (int k = 0; k < 4; ++k) out->quarter[k] = p.q[k];
    out->digit_bits = p.D;
  }
  out->records_left = uint64_t(1) << (out->quarter[0] + out->quarter[2]);
  out->records_right = uint64_t(1) << (out->quarter[1] + out->quarter[3]);
  out->device_bytes = footprint_estimate(m, n, 0);
  return MSP_OK;
}

const char *msp_device_name(void) {
  thread_local std::string name;
  name.clear();
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess)
    name = prop.name;
  else
    cudaGetLastError();
  return name.c_str();
}

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

int msp_set_option(msp_instance *inst, int option, int64_t value) {
  if (!inst) return fail(MSP_EINVAL, "null instance");
  switch (option) {
    case MSP_OPT_EXACT_PATH:
      inst->force_exact = value != 0;
      return MSP_OK;
    case MSP_OPT_CLASS_PART:
      if (value < 0) return fail(MSP_EINVAL, "class part must be >= 0");
      inst->part = value;
      return MSP_OK;
    case MSP_OPT_CLASS_PARTS:
      if (value < 1) return fail(MSP_EINVAL, "class parts must be >= 1");
      inst->parts = value;
      return MSP_OK;
    case MSP_OPT_CLASS_BITS:
      if (value < -1 || value > kMaxStreamClassBits) return fail(MSP_ERANGE, "class bits must lie in [-1, 27]");
      inst->plan_B = static_cast<int>(value);
      return MSP_OK;
    case MSP_OPT_DIGIT_BITS:
      if (value < -1 || value > 12) return fail(MSP_ERANGE, "digit bits must lie in [-1, 12]");
      inst->plan_D = static_cast<int>(value);
      return MSP_OK;
    case MSP_OPT_INNER_BITS:
      if (value < -1 || value > 12) return fail(MSP_ERANGE, "inner bits must lie in [-1, 12]");
      inst->plan_inner = static_cast<int>(value);
      return MSP_OK;
    case MSP_OPT_DIRECT:
      if (value < -1 || value > 1) return fail(MSP_ERANGE, "direct must be -1, 0 or 1");
      inst->direct = static_cast<int>(value);
      return MSP_OK;
    case MSP_OPT_FIRST:
      if (value < 0 || value > 1) return fail(MSP_ERANGE, "first must be 0 or 1");
      inst->first_only = value != 0;
      return MSP_OK;
    case MSP_OPT_WAIT_LIMIT_US:
      if (value < 1 || value > 60000000) return fail(MSP_ERANGE, "wait limit must lie in [1, 6e7] us");
      inst->wait_ns = static_cast<uint64_t>(value) * 1000u;
      return MSP_OK;
    case MSP_OPT_WAIT_CHECK:
      if (value < 0 || value > 1) return fail(MSP_ERANGE, "wait check must be 0 or 1");
      inst->wait_check = static_cast<int>(value);
      return MSP_OK;
    case MSP_OPT_TABLE_BITS:
      if (value != -1 && (value < 12 || value > 15)) return fail(MSP_ERANGE, "table bits must be -1 or lie in [12, 15]");
      inst->table_bits = static_cast<int>(value);
      return MSP_OK;
    default:
      return fail(MSP_EINVAL, "unknown option");
  }
}

int msp_set_profiling(msp_instance *inst, int on) {
  if (!inst) return fail(MSP_EINVAL, "null instance");
  inst->profiling = on != 0;
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
  return msp_solve_batch_path(A, d, m, n, count, -1, masks, offsets);
}

int msp_solve_batch_path(const int32_t *const *A, const int32_t *const *d, int m, int n, int count, int path,
                         uint64_t **masks, size_t *offsets) {
  if (!A || !d || !masks || !offsets || count < 0) return fail(MSP_EINVAL, "null argument");
  if (path < -1 || path > 1) return fail(MSP_ERANGE, "path must be -1, 0 or 1");
  *masks = nullptr;
  offsets[0] = 0;
  for (int k = 0; k < count; ++k) {
    const int rc = validate(A[k], d[k], m, n);
    if (rc != MSP_OK) return rc;
  }
  if (count == 0) return MSP_OK;
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1)
    return fail(MSP_ECUDA, "no CUDA device available");
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
    return fail(MSP_ECUDA, "cudaStreamCreate failed");
  std::vector<std::vector<uint64_t>> raw;
  int rc = msp::kDirectFallback;
  if (path != 0) {
    msp_instance probe;  // only for the memory budget of the device
    cudaGetDevice(&probe.device);
    rc = msp::solve_batch_direct(A, d, m, n, count, raw, s, msp::solve_budget(&probe, 0));
    if (rc == msp::kDirectFallback && path == 1) rc = fail(MSP_ERANGE, "the batch does not fit the direct pass");
  }
  if (rc == msp::kDirectFallback) rc = msp::solve_batch_impl(A, d, m, n, count, raw, s, 0);
  cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  if (rc != MSP_OK) return rc;
  // sort and de-duplicate each instance's masks (most significant word first)
  const int W = (n + 63) / 64;
  std::vector<uint64_t> all;
  for (int k = 0; k < count; ++k) {
    const size_t cnt = raw[k].size() / 2;
    std::vector<std::pair<uint64_t, uint64_t>> v(cnt);
    for (size_t i = 0; i < cnt; ++i) v[i] = {raw[k][2 * i + 1], raw[k][2 * i]};
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    for (auto &x : v) {
      all.push_back(x.second);
      if (W > 1) all.push_back(x.first);
    }
    offsets[k + 1] = offsets[k] + v.size();
  }
  if (!all.empty()) {
    *masks = static_cast<uint64_t *>(std::malloc(sizeof(uint64_t) * all.size()));
    if (!*masks) return fail(MSP_ENOMEM, "host allocation failed");
    std::memcpy(*masks, all.data(), sizeof(uint64_t) * all.size());
  }
  return MSP_OK;
}

}  // extern "C"
