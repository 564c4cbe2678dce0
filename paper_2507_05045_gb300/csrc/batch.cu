// msp_solve_batch: many instances of one (m, n) solved together.
//
// Every instance gets its quarter lists and class buckets (S1, S2) as in a
// single solve; then each residue pass runs ONE scatter launch and ONE join
// launch over the work units (instance, side, class, slice) of all
// instances: the streaming kernels walk a device table of instances, so a
// batch of small instances fills the GPU that one of them would leave idle.
// Matches carry instance * M + class; they are split by instance for the
// exact recovery and all-row verification (S6).  An instance whose classes
// do not fit the streaming partitions, or a pass that overflows, is solved
// again on its own by the single-instance path, so the result never depends
// on the fast path succeeding.
#include "host_internal.h"
#include "host_util.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace msp {

namespace {

struct BatchItem {
  int idx = 0;  // position in the caller's arrays
  InstanceConst ic{};
  QuarterDev qd[4];
  BucketDev bd[4];
  SideGen gens[2];
  std::vector<unsigned long long> csz[2];
  std::vector<uint32_t> capv[2];
  std::vector<uint64_t> base_h[2];
  uint64_t *d_base[2] = {nullptr, nullptr};
  uint32_t *d_cap[2] = {nullptr, nullptr};
  bool alone = false;  // solved on its own by the single-instance path
};

// Quarter element recovery and exact verification of the matches of one
// instance (keys and classes already on the device); raw solution masks
// (two words each) are appended to `out`.
int recover_and_verify(const BatchItem &it, uint32_t cmask, const uint64_t *d_key, const uint32_t *d_cls,
                       uint64_t nmatch, DevAlloc &da, cudaStream_t s, std::vector<uint64_t> &out) {
  RecoverDev rd{};
  rd.match_key = d_key;
  rd.match_cls = d_cls;
  rd.nmatch = nmatch;
  rd.side[0] = it.gens[0];
  rd.side[1] = it.gens[1];
  rd.oidx[0] = it.bd[0].idx;
  rd.iidx[0] = it.bd[1].idx;
  rd.oidx[1] = it.bd[2].idx;
  rd.iidx[1] = it.bd[3].idx;
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
  vd.ic = it.ic;
  for (int k = 0; k < 4; ++k) {
    vd.qvec[k] = it.qd[k].vec;
    vd.qsize[k] = it.qd[k].size;
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
    if (hc[0] <= cap) {
      const size_t old = out.size();
      out.resize(old + 2 * hc[0]);
      if (hc[0]) {
        CK(cudaMemcpyAsync(out.data() + old, vd.sol, sizeof(uint64_t) * 2 * hc[0], cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
      }
      return MSP_OK;
    }
    if (hc[0] > (1ull << 28)) return fail(MSP_EOVERFLOW, "more than 2^28 solutions");
    cap = hc[0];
  }
  return MSP_OK;
}

}  // namespace

// Solve instances A[k], d[k] (k < count) of one (m, n).  raw[k] receives the
// unsorted two-word solution masks of instance k.  `alone` solves use their
// own msp_instance on the same stream.
int solve_batch_impl(const int32_t *const *A, const int32_t *const *d, int m, int n, int count,
                     std::vector<std::vector<uint64_t>> &raw, cudaStream_t s, size_t budget_cap) {
  raw.assign(count, {});
  const Plan p = make_plan(m, n);
  const uint32_t M = 1u << p.B, cmask = M - 1u;
  const int nd = 1 << p.D;
  DevAlloc da(s);

  // ---- items: feasible right-hand sides only ----
  std::vector<BatchItem> items;
  for (int k = 0; k < count; ++k) {
    bool feasible = true;
    for (int i = 0; i < m && feasible; ++i) {
      int64_t rs = 0;
      for (int j = 0; j < n; ++j) rs += A[k][(size_t)i * n + j];
      feasible = d[k][i] <= rs;
    }
    if (!feasible) continue;
    BatchItem it;
    it.idx = k;
    items.push_back(std::move(it));
  }
  const int K = static_cast<int>(items.size());
  if (K == 0) return MSP_OK;

  // ---- S0: constants and packed columns of every instance, one upload ----
  std::vector<uint64_t> pcol((size_t)K * n * kMaxVecWords, 0), kcol((size_t)K * n);
  std::vector<uint32_t> ccol((size_t)K * n);
  std::vector<int64_t> col(m), dv(m);
  for (int t = 0; t < K; ++t) {
    BatchItem &it = items[t];
    const int32_t *Ak = A[it.idx];
    InstanceConst &ic = it.ic;
    ic.m = m;
    ic.n = n;
    ic.W = p.W;
    for (int q = 0; q < 4; ++q) {
      ic.q[q] = p.q[q];
      ic.col0[q] = p.col0[q];
    }
    for (int i = 0; i < kMaxRows; ++i) ic.w_row[i] = p.w_row[i];
    for (int i = 0; i < kMaxClassRows; ++i) ic.c_row[i] = p.c_row[i];
    ic.t_rows = p.t;
    ic.class_bits = p.B;
    for (int j = 0; j < n; ++j) {
      uint32_t c = 0;
      for (int i = 0; i < m; ++i) {
        col[i] = Ak[(size_t)i * n + j];
        pcol[((size_t)t * n + j) * kMaxVecWords + i / 4] |= static_cast<uint64_t>(col[i]) << (16 * (i % 4));
      }
      kcol[(size_t)t * n + j] = key_of(p, col.data());
      for (int i = 0; i < p.t; ++i) c += p.c_row[i] * static_cast<uint32_t>(col[i]);
      ccol[(size_t)t * n + j] = c;
    }
    for (int i = 0; i < m; ++i) {
      dv[i] = d[it.idx][i];
      ic.dvec[i / 4] |= static_cast<uint64_t>(dv[i]) << (16 * (i % 4));
    }
    ic.kd = key_of(p, dv.data());
    ic.cd = class_of(p, dv.data());
  }
  uint64_t *d_pcol, *d_kcol;
  uint32_t *d_ccol;
  CK(da.get(&d_pcol, pcol.size()));
  CK(da.get(&d_kcol, kcol.size()));
  CK(da.get(&d_ccol, ccol.size()));
  CK(cudaMemcpyAsync(d_pcol, pcol.data(), pcol.size() * 8, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_kcol, kcol.data(), kcol.size() * 8, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_ccol, ccol.data(), ccol.size() * 4, cudaMemcpyHostToDevice, s));

  // ---- S1, S2 per instance: quarter lists, class buckets, class sizes ----
  const int qk[4] = {0, 2, 1, 3};
  const int64_t mul[4] = {1, 1, -1, -1};
  uint32_t *d_hist, *d_cursor, *d_scantmp;
  CK(da.get(&d_hist, M));
  CK(da.get(&d_cursor, (size_t)M + 1));
  CK(da.get(&d_scantmp, ((size_t)M + 1 + 4095) / 4096 + 1));
  unsigned long long *d_csz;
  CK(da.get(&d_csz, (size_t)K * 2 * M));
  for (int t = 0; t < K; ++t) {
    BatchItem &it = items[t];
    for (int q = 0; q < 4; ++q) {
      it.qd[q].q = p.q[q];
      it.qd[q].size = int64_t(1) << p.q[q];
      CK(da.get(&it.qd[q].vec, (size_t)p.W * it.qd[q].size));
      CK(da.get(&it.qd[q].key, it.qd[q].size));
      CK(da.get(&it.qd[q].cls, it.qd[q].size));
      CK(da.get(&it.qd[q].v1, it.qd[q].size));
      CK(launch_gray(it.ic, d_pcol + (size_t)t * n * kMaxVecWords, d_kcol + (size_t)t * n,
                     d_ccol + (size_t)t * n, it.qd[q], p.col0[q], s));
    }
    const uint64_t kadd[4] = {0, 0, it.ic.kd, 0};
    const uint32_t cadd[4] = {0, 0, it.ic.cd, 0};
    for (int l = 0; l < 4; ++l) {
      const QuarterDev &q = it.qd[qk[l]];
      BucketDev &b = it.bd[l];
      b.size = q.size;
      CK(da.get(&b.key, q.size));
      CK(da.get(&b.cls, q.size));
      CK(da.get(&b.idx, q.size));
      CK(da.get(&b.off, (size_t)M + 1));
      CK(cudaMemsetAsync(d_hist, 0, sizeof(uint32_t) * M, s));
      CK(launch_count_classes(q.cls, q.size, static_cast<uint32_t>(mul[l]), cadd[l], cmask, d_hist, s));
      CK(launch_scan_u32(d_hist, b.off, M, d_scantmp, s));
      CK(cudaMemcpyAsync(d_cursor, b.off, sizeof(uint32_t) * M, cudaMemcpyDeviceToDevice, s));
      CK(launch_bucket_scatter(q, mul[l], kadd[l], cadd[l], cmask, d_cursor, b, s));
    }
    for (int side = 0; side < 2; ++side) {
      const BucketDev &o = it.bd[side == 0 ? 0 : 2];
      const BucketDev &in = it.bd[side == 0 ? 1 : 3];
      SideGen &g = it.gens[side];
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
      unsigned long long *dst = d_csz + ((size_t)t * 2 + side) * M;
      if (o.size < (int64_t)M)  // fewer outer elements than classes: sum over the elements
        CK(launch_class_sizes_elems(o.cls, o.size, in.off, M, 0, M, dst, s));
      else
        CK(launch_class_sizes(o.off, in.off, M, 0, M, dst, s));
    }
  }
  std::vector<unsigned long long> csz_all((size_t)K * 2 * M);
  CK(cudaMemcpyAsync(csz_all.data(), d_csz, sizeof(unsigned long long) * csz_all.size(), cudaMemcpyDeviceToHost,
                     s));
  CK(cudaStreamSynchronize(s));

  // ---- partition capacities; an instance with an oversized class goes alone ----
  std::vector<int> fast_items;
  for (int t = 0; t < K; ++t) {
    BatchItem &it = items[t];
    for (int side = 0; side < 2; ++side) {
      it.csz[side].assign(csz_all.begin() + ((size_t)t * 2 + side) * M,
                          csz_all.begin() + ((size_t)t * 2 + side + 1) * M);
      it.capv[side].assign(M, 0);
      for (uint32_t c = 0; c < M; ++c) {
        const double mean = (double)it.csz[side][c] / nd;
        uint64_t cap = static_cast<uint64_t>(std::ceil(mean + 7.0 * std::sqrt(mean) + 32.0));
        cap = std::min<uint64_t>((cap + 15) & ~uint64_t(15), kFastCap);
        const bool fits = mean + 4.0 * std::sqrt(mean) <= (double)kFastCap;
        if (!fits) it.alone = true;
        it.capv[side][c] = static_cast<uint32_t>(cap);
      }
    }
    if (!it.alone) fast_items.push_back(t);
  }

  // ---- residue passes: classes [c0, c1) of every fast instance per pass ----
  const int KF = static_cast<int>(fast_items.size());
  bool redo_all = false;
  std::vector<std::vector<uint64_t>> mkeys(K);
  std::vector<std::vector<uint32_t>> mcls(K);
  if (KF > 0) {
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    cudaMemPool_t pool;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t reserved = 0, used = 0;
      cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved);
      cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used);
      if (reserved > used) free_b += reserved - used;
    }
    const double avail = (double)free_b;
    double budget = budget_cap ? (double)budget_cap - (double)da.bytes : 0.85 * avail;
    budget = std::min(budget, 0.95 * avail) - (double)(64 << 20);
    struct PassPlan {
      uint32_t c0, c1;
    };
    std::vector<PassPlan> plan;
    for (int f = 0; f < KF; ++f) {
      BatchItem &it = items[fast_items[f]];
      it.base_h[0].assign(M, 0);
      it.base_h[1].assign(M, 0);
    }
    uint64_t need[2] = {0, 0};
    for (uint32_t c0 = 0; c0 < M;) {
      uint64_t acc[2] = {0, 0};
      uint32_t c = c0;
      while (c < M) {
        uint64_t add[2] = {0, 0};
        for (int f = 0; f < KF; ++f)
          for (int side = 0; side < 2; ++side) add[side] += (uint64_t)items[fast_items[f]].capv[side][c] * nd;
        if (c > c0 && 8.0 * (double)(acc[0] + add[0] + acc[1] + add[1]) > budget) break;
        // regions: instance-major inside the class
        for (int f = 0; f < KF; ++f)
          for (int side = 0; side < 2; ++side) {
            BatchItem &it = items[fast_items[f]];
            it.base_h[side][c] = acc[side];
            acc[side] += (uint64_t)it.capv[side][c] * nd;
          }
        ++c;
      }
      plan.push_back({c0, c});
      need[0] = std::max(need[0], acc[0]);
      need[1] = std::max(need[1], acc[1]);
      c0 = c;
    }
    if (8.0 * (double)(need[0] + need[1]) > budget + (64 << 20))
      return fail(MSP_ENOMEM, "batch: memory budget too small for one residue class of every instance");
    uint64_t *rec[2];
    CK(da.get(&rec[0], need[0]));
    CK(da.get(&rec[1], need[1]));
    int max_c = 0;
    for (auto &pp : plan) max_c = std::max<int>(max_c, pp.c1 - pp.c0);
    uint32_t *d_fill[2];
    CK(da.get(&d_fill[0], (size_t)KF * max_c * nd));
    CK(da.get(&d_fill[1], (size_t)KF * max_c * nd));
    std::vector<FastInst> tab(KF);
    for (int f = 0; f < KF; ++f) {
      BatchItem &it = items[fast_items[f]];
      for (int side = 0; side < 2; ++side) {
        CK(da.get(&it.d_base[side], M));
        CK(da.get(&it.d_cap[side], M));
        CK(cudaMemcpyAsync(it.d_base[side], it.base_h[side].data(), sizeof(uint64_t) * M, cudaMemcpyHostToDevice,
                           s));
        CK(cudaMemcpyAsync(it.d_cap[side], it.capv[side].data(), sizeof(uint32_t) * M, cudaMemcpyHostToDevice, s));
        tab[f].side[side] = it.gens[side];
        tab[f].class_base[side] = it.d_base[side];
        tab[f].cap[side] = it.d_cap[side];
        tab[f].fill[side] = d_fill[side] + (size_t)f * max_c * nd;
      }
      tab[f].tag = static_cast<uint32_t>(f) * M;
    }
    FastInst *d_tab;
    CK(da.get(&d_tab, KF));
    CK(cudaMemcpyAsync(d_tab, tab.data(), sizeof(FastInst) * KF, cudaMemcpyHostToDevice, s));
    const uint64_t match_cap = 1u << 20;
    uint64_t *match_key;
    uint32_t *match_cls;
    unsigned long long *match_count;
    unsigned int *d_flags;  // [0] timeout, [1 + f] overflow of fast instance f
    CK(da.get(&match_key, match_cap));
    CK(da.get(&match_cls, match_cap));
    CK(da.get(&match_count, 1));
    CK(da.get(&d_flags, 1 + (size_t)KF));
    CK(cudaMemsetAsync(match_count, 0, sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(d_flags, 0, sizeof(unsigned int) * (1 + (size_t)KF), s));
    FastPass fp{};
    fp.inst = d_tab;
    fp.ninst = KF;
    fp.slices[0] = items[fast_items[0]].gens[0].slices;
    fp.slices[1] = items[fast_items[0]].gens[1].slices;
    fp.cmask = cmask;
    fp.D = p.D;
    fp.S = p.S;
    fp.rec[0] = rec[0];
    fp.rec[1] = rec[1];
    fp.overflow = d_flags + 1;
    fp.error = d_flags;
    fp.wait_ns = kDefaultWaitNs;
    fp.wait_check = 0;
    fp.match_key = match_key;
    fp.match_cls = match_cls;
    fp.match_count = match_count;
    fp.match_cap = match_cap;
    for (const PassPlan &pp : plan) {
      const int run = static_cast<int>(pp.c1 - pp.c0);
      fp.c0 = static_cast<int>(pp.c0);
      fp.nclass = run;
      for (int side = 0; side < 2; ++side)
        CK(cudaMemsetAsync(d_fill[side], 0, sizeof(uint32_t) * (size_t)KF * max_c * nd, s));
      CK(launch_scatter_fast(fp, run, s));
      CK(launch_join_fast(fp, run, s));
    }
    std::vector<unsigned int> flags(1 + (size_t)KF);
    unsigned long long nmatch = 0;
    CK(cudaMemcpyAsync(flags.data(), d_flags, sizeof(unsigned int) * flags.size(), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&nmatch, match_count, sizeof(nmatch), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (flags[0]) return fail(MSP_ETIMEDOUT, "a bulk copy did not complete within its time limit");
    for (int f = 0; f < KF; ++f)
      if (flags[1 + f]) items[fast_items[f]].alone = true;  // a partition overflowed: solve it alone
    if (nmatch > match_cap) {
      redo_all = true;
    } else if (nmatch) {
      std::vector<uint64_t> hk(nmatch);
      std::vector<uint32_t> hc(nmatch);
      CK(cudaMemcpyAsync(hk.data(), match_key, sizeof(uint64_t) * nmatch, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(hc.data(), match_cls, sizeof(uint32_t) * nmatch, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (uint64_t i = 0; i < nmatch; ++i) {
        const int t = fast_items[hc[i] / M];
        mkeys[t].push_back(hk[i]);
        mcls[t].push_back(hc[i] % M);
      }
    }
    // the pass buffers are no longer needed
    da.free1(rec[0], sizeof(uint64_t) * need[0]);
    da.free1(rec[1], sizeof(uint64_t) * need[1]);
  }

  // ---- S6 per instance with matches ----
  if (!redo_all) {
    for (int t = 0; t < K; ++t) {
      if (items[t].alone || mkeys[t].empty()) continue;
      const uint64_t nm = mkeys[t].size();
      uint64_t *dk;
      uint32_t *dc;
      CK(da.get(&dk, nm));
      CK(da.get(&dc, nm));
      CK(cudaMemcpyAsync(dk, mkeys[t].data(), sizeof(uint64_t) * nm, cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync(dc, mcls[t].data(), sizeof(uint32_t) * nm, cudaMemcpyHostToDevice, s));
      const int rc = recover_and_verify(items[t], cmask, dk, dc, nm, da, s, raw[items[t].idx]);
      if (rc != MSP_OK) return rc;
    }
  }
  da.release();
  CK(cudaStreamSynchronize(s));

  // ---- instances the streaming batch could not take: single-instance path ----
  for (int t = 0; t < K; ++t) {
    if (!(redo_all || items[t].alone)) continue;
    msp_instance inst;
    inst.m = m;
    inst.n = n;
    inst.A.assign(A[items[t].idx], A[items[t].idx] + (size_t)m * n);
    inst.d.assign(d[items[t].idx], d[items[t].idx] + m);
    inst.stream = s;
    inst.own_stream = false;
    cudaGetDevice(&inst.device);
    uint64_t *mk = nullptr;
    size_t c = 0;
    int words = 1;
    const int rc = solve_instance(&inst, &mk, &c, &words);
    if (rc != MSP_OK) return rc;
    std::vector<uint64_t> &out = raw[items[t].idx];
    for (size_t i = 0; i < c; ++i) {
      out.push_back(mk[(size_t)words * i]);
      out.push_back(words > 1 ? mk[(size_t)words * i + 1] : 0);
    }
    msp_free_solutions(mk);
  }
  return MSP_OK;
}

}  // namespace msp
