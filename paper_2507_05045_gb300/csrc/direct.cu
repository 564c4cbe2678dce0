// Direct pass of libmsp, host side: the plan, the lists of an instance (or a
// batch of instances), the launches of the class joins and the
// verification, and the solves built from them (direct_join.cu and
// direct_kernels.cu hold the kernels).
#include "direct_internal.cuh"
#include "host_internal.h"
#include "host_util.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace msp {

// -------------------------------------------------------------------------
// Host side.
// -------------------------------------------------------------------------
DirectPlan make_direct_plan(int m, int n, int table_bits) {
  DirectPlan d{};
  d.m = m;
  d.n = n;
  d.W = (m + 3) / 4;
  d.cols[0] = (n + 1) / 2;
  d.cols[1] = n - d.cols[0];
  const int lg = std::max(d.cols[0], d.cols[1]);
  // about 2^13 records per class and side; inner buckets of about 16
  d.B = std::max(0, lg - 13);
  d.TB = table_bits >= 12 && table_bits <= 15 ? table_bits : 14;
  for (int s = 0; s < 2; ++s) {
    const int c = d.cols[s];
    int qi = std::min(c, d.B + 4);
    int qo = c - qi;
    if (qo > 9) {  // small halves: everything beyond 9 outer columns goes inner
      qo = 9;
      qi = c - qo;
    }
    d.qo[s] = qo;
    d.qi[s] = qi;
  }
  d.col_o[0] = 0;
  d.col_i[0] = d.qo[0];
  d.col_o[1] = d.cols[0];
  d.col_i[1] = d.cols[0] + d.qo[1];
  d.t = std::min(m, d.B <= 6 ? 1 : (d.B <= 14 ? 2 : (d.B <= 21 ? 3 : 4)));
  d.ok = n >= 2 && d.qi[0] <= kInnerMax && d.qi[1] <= kInnerMax && (1 << d.qo[0]) <= kOuterMax &&
         (1 << d.qo[1]) <= kOuterMax && d.B <= 27;
  return d;
}

size_t direct_footprint(const DirectPlan &d) {
  double b = 0;
  for (int s = 0; s < 2; ++s) b += 8.0 * std::ldexp(1.0, d.qi[s]);  // inner keys and masks
  b += 2.0 * 4.0 * (std::ldexp(1.0, d.B) + 1);                       // bucket offsets
  b += 4.0 * (std::ldexp(1.0, d.B) + 1);                             // counts / cursors while building
  b += 16.0 * std::ldexp(1.0, std::max(d.qi[0], d.qi[1]) - kHighMax) + 4096;  // low subsets while building
  b += 8.0 * (std::ldexp(1.0, d.B) + 1) + 8.0 * (1 << kHighMax);     // coarse buckets, high subsets
  b += 12.0 * kDirectMatchCap + (64 << 20);                          // matches, small tables, margin
  return static_cast<size_t>(b);
}

namespace {

// Host and device lists of one instance of a direct pass.
struct DirectLists {
  int no[2] = {0, 0};  // outer subsets per side
  uint64_t dvec[4] = {0, 0, 0, 0};
  uint32_t *ikey[2] = {nullptr, nullptr}, *imask[2] = {nullptr, nullptr}, *ioff[2] = {nullptr, nullptr};
  uint64_t *icol[2] = {nullptr, nullptr};
  uint32_t *d_okey[2] = {nullptr, nullptr}, *d_ocls[2] = {nullptr, nullptr}, *d_omask[2] = {nullptr, nullptr};
  uint64_t *d_ovec[2] = {nullptr, nullptr};
};

struct Copier {
  msp_stats *st;
  cudaStream_t s;
  cudaError_t h2d(void *dst, const void *src, size_t b) {
    if (st) st->h2d_bytes += b;
    return cudaMemcpyAsync(dst, src, b, cudaMemcpyHostToDevice, s);
  }
  cudaError_t d2h(void *dst, const void *src, size_t b) {
    if (st) st->d2h_bytes += b;
    return cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToHost, s);
  }
};

// S0 on the host for one instance: the column keys and classes, the packed
// right-hand side, the column tables of the outer quarters o[side] (their
// lists are built on the device) and of the inner quarters g[side], and the
// packed column vectors icol[side] of the inner quarters.
void prep_direct_host(const int32_t *A, const int32_t *d, int m, int n, const DirectPlan &dp, const Plan &kp,
                      DirectLists &L, OuterSeg o[2], InnerGen g[2], std::vector<uint64_t> icol[2]) {
  const uint32_t M = 1u << dp.B, cmask = M - 1u;
  std::vector<uint32_t> ck(n), cc(n);
  std::vector<uint64_t> pc((size_t)n * 4, 0);
  for (int j = 0; j < n; ++j) {
    uint32_t k = 0, c = 0;
    for (int i = 0; i < m; ++i) {
      const uint32_t a = static_cast<uint32_t>(A[(size_t)i * n + j]);
      k += static_cast<uint32_t>(kp.w_row[i]) * a;
      if (i < dp.t) c += kp.c_row[i] * a;
      pc[(size_t)j * 4 + i / 4] += static_cast<uint64_t>(a) << (16 * (i % 4));
    }
    ck[j] = k;
    cc[j] = c;
  }
  uint32_t kd = 0, cd = 0;
  for (int i = 0; i < m; ++i) {
    const uint32_t di = static_cast<uint32_t>(d[i]);
    kd += static_cast<uint32_t>(kp.w_row[i]) * di;
    if (i < dp.t) cd += kp.c_row[i] * di;
    L.dvec[i / 4] += static_cast<uint64_t>(di) << (16 * (i % 4));
  }
  for (int sd = 0; sd < 2; ++sd) {
    const int q = dp.qo[sd], c0 = dp.col_o[sd];
    L.no[sd] = 1 << q;
    o[sd] = OuterSeg{};
    for (int j = 0; j < q; ++j) {
      o[sd].ck[j] = ck[c0 + j];
      o[sd].cc[j] = cc[c0 + j];
      for (int w = 0; w < 4; ++w) o[sd].pc[j][w] = pc[(size_t)(c0 + j) * 4 + w];
    }
    o[sd].q = q;
    o[sd].neg = sd;
    o[sd].kd = kd;
    o[sd].cd = cd;
    o[sd].cmask = cmask;
  }
  for (int sd = 0; sd < 2; ++sd) {
    const int q = dp.qi[sd], c0 = dp.col_i[sd];
    g[sd] = InnerGen{};
    for (int j = 0; j < q; ++j) {
      g[sd].ck[j] = ck[c0 + j];
      g[sd].cc[j] = cc[c0 + j];
    }
    g[sd].q = q;
    g[sd].neg = sd;
    g[sd].cmask = cmask;
    icol[sd].assign(pc.begin() + (size_t)c0 * 4, pc.begin() + (size_t)(c0 + q) * 4);
    icol[sd].resize((size_t)std::max(q, 1) * 4, 0);
  }
}

// S0 + S1 + S2 of one instance: host preparation, then the inner lists
// bucketed by class on the device: the low subsets by coarse class and the
// high subsets, then class counts by windows, bucket starts and placement
// by windows.  `cnt` and `scantmp` are
// scratch of 2^B + 1 and (2^B + 1) / 4096 + 1 entries, shared by successive
// calls.
int build_direct_lists(const int32_t *A, const int32_t *d, int m, int n, const DirectPlan &dp, const Plan &kp,
                       DevAlloc &da, Copier &cp, Prof &prof, uint32_t *cnt, uint32_t *scantmp, DirectLists &L) {
  cudaStream_t s = cp.s;
  const uint32_t M = 1u << dp.B;
  InnerGen gs[2];
  OuterSeg os[2];
  std::vector<uint64_t> icol[2];
  prep_direct_host(A, d, m, n, dp, kp, L, os, gs, icol);
  for (int sd = 0; sd < 2; ++sd) {
    const int q = dp.qi[sd];
    const uint64_t ni = uint64_t(1) << q;
    CK(da.get(&L.ikey[sd], ni));
    CK(da.get(&L.imask[sd], ni));
    CK(da.get(&L.ioff[sd], (size_t)M + 1));
    CK(da.get(&L.icol[sd], icol[sd].size()));
    CK(cp.h2d(L.icol[sd], icol[sd].data(), sizeof(uint64_t) * icol[sd].size()));
  }
  for (int sd = 0; sd < 2; ++sd) {
    const int q = dp.qi[sd];
    WinBuild w{};
    w.B = dp.B;
    w.cmask = M - 1u;
    w.hq = std::min(q, kHighMax);
    w.h = q - w.hq;
    w.logW = std::min(kWinBits, dp.B);
    w.gshift = std::max(0, w.logW - 2);
    w.nc = 1u << (dp.B - w.gshift);
    const size_t nl = size_t(1) << w.h;
    uint4 *low;
    uint32_t *lcur, *loff, *hkey, *hcls;
    CK(da.get(&low, nl));
    CK(da.get(&lcur, (size_t)w.nc + 1));
    CK(da.get(&loff, (size_t)w.nc + 1));
    CK(da.get(&hkey, size_t(1) << w.hq));
    CK(da.get(&hcls, size_t(1) << w.hq));
    InnerGen gl = gs[sd];
    gl.q = w.h;
    CK(cudaMemsetAsync(lcur, 0, sizeof(uint32_t) * w.nc, s));
    LAUNCH(MSP_K_BUCKET, 1, 0, launch_win_low(gl, w.gshift, lcur, nullptr, s));
    LAUNCH(MSP_K_BUCKET, 3, 0, launch_scan_u32(lcur, loff, w.nc, scantmp, s));
    CK(cudaMemcpyAsync(lcur, loff, sizeof(uint32_t) * w.nc, cudaMemcpyDeviceToDevice, s));
    LAUNCH(MSP_K_BUCKET, 1, 0, launch_win_low(gl, w.gshift, lcur, low, s));
    LAUNCH(MSP_K_BUCKET, 1, 0, launch_win_high(gs[sd], w.h, w.hq, hkey, hcls, s));
    w.low = low;
    w.loff = loff;
    w.hkey = hkey;
    w.hcls = hcls;
    w.cnt = cnt;
    LAUNCH(MSP_K_BUCKET, 1, 0, launch_win(w, false, s));
    LAUNCH(MSP_K_BUCKET, 3, 0, launch_scan_u32(cnt, L.ioff[sd], M, scantmp, s));
    w.ioff = L.ioff[sd];
    w.ikey = L.ikey[sd];
    w.imask = L.imask[sd];
    LAUNCH(MSP_K_BUCKET, 1, 0, launch_win(w, true, s));
    da.free1(hcls, sizeof(uint32_t) << w.hq);
    da.free1(hkey, sizeof(uint32_t) << w.hq);
    da.free1(loff, sizeof(uint32_t) * ((size_t)w.nc + 1));
    da.free1(lcur, sizeof(uint32_t) * ((size_t)w.nc + 1));
    da.free1(low, sizeof(uint4) * nl);
  }
  // S1 of the outer quarters on the device
  for (int sd = 0; sd < 2; ++sd) {
    const size_t no = static_cast<size_t>(L.no[sd]);
    CK(da.get(&L.d_okey[sd], no));
    CK(da.get(&L.d_ocls[sd], no));
    CK(da.get(&L.d_omask[sd], no));
    CK(da.get(&L.d_ovec[sd], no * 4));
    os[sd].okey = L.d_okey[sd];
    os[sd].ocls = L.d_ocls[sd];
    os[sd].omask = L.d_omask[sd];
    os[sd].ovec = L.d_ovec[sd];
  }
  OuterSeg *d_os;
  CK(da.get(&d_os, 2));
  CK(cp.h2d(d_os, os, sizeof(OuterSeg) * 2));
  LAUNCH(MSP_K_GRAY, 1, 0, launch_direct_outer(d_os, 2, s));
  return MSP_OK;
}

// The lists of the instances idx[k] of a batch (all of one (m, n)), built
// together: the host part per instance, then one upload per array kind and,
// per side, one count launch, one offsets launch (one block per instance)
// and one placement launch over the inner quarters of all instances.
int build_direct_lists_batch(const int32_t *const *A, const int32_t *const *d, const std::vector<int> &idx, int m,
                             int n, const DirectPlan &dp, const Plan &kp, DevAlloc &da, Copier &cp, Prof &prof,
                             std::vector<DirectLists> &lists) {
  cudaStream_t s = cp.s;
  const size_t K = idx.size();
  const uint32_t M = 1u << dp.B;
  lists.assign(K, DirectLists{});
  std::vector<InnerSeg> segs(2 * K);  // segment side * K + k
  std::vector<OuterSeg> osegs(2 * K);
  std::vector<uint64_t> icol_h[2];
  for (size_t k = 0; k < K; ++k) {
    InnerGen g[2];
    OuterSeg o[2];
    std::vector<uint64_t> icol[2];
    prep_direct_host(A[idx[k]], d[idx[k]], m, n, dp, kp, lists[k], o, g, icol);
    for (int sd = 0; sd < 2; ++sd) {
      segs[sd * K + k].g = g[sd];
      osegs[sd * K + k] = o[sd];
      icol_h[sd].insert(icol_h[sd].end(), icol[sd].begin(), icol[sd].end());
    }
  }
  for (int sd = 0; sd < 2; ++sd) {
    const uint64_t ni = uint64_t(1) << dp.qi[sd];
    const size_t no = size_t(1) << dp.qo[sd];
    const size_t nic = icol_h[sd].size() / K;
    uint32_t *ikey, *imask, *ioff, *cnt, *okey, *ocls, *omask;
    uint64_t *icol, *ovec;
    CK(da.get(&ikey, ni * K));
    CK(da.get(&imask, ni * K));
    CK(da.get(&ioff, ((size_t)M + 1) * K));
    CK(da.get(&cnt, (size_t)M * K));
    CK(da.get(&icol, icol_h[sd].size()));
    CK(da.get(&okey, no * K));
    CK(da.get(&ocls, no * K));
    CK(da.get(&omask, no * K));
    CK(da.get(&ovec, 4 * no * K));
    CK(cp.h2d(icol, icol_h[sd].data(), 8 * icol_h[sd].size()));
    CK(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * M * K, s));
    for (size_t k = 0; k < K; ++k) {
      DirectLists &L = lists[k];
      L.ikey[sd] = ikey + ni * k;
      L.imask[sd] = imask + ni * k;
      L.ioff[sd] = ioff + ((size_t)M + 1) * k;
      L.icol[sd] = icol + nic * k;
      L.d_okey[sd] = okey + no * k;
      L.d_ocls[sd] = ocls + no * k;
      L.d_omask[sd] = omask + no * k;
      L.d_ovec[sd] = ovec + 4 * no * k;
      OuterSeg &O = osegs[sd * K + k];
      O.okey = L.d_okey[sd];
      O.ocls = L.d_ocls[sd];
      O.omask = L.d_omask[sd];
      O.ovec = L.d_ovec[sd];
      InnerSeg &S = segs[sd * K + k];
      S.cnt = cnt + (size_t)M * k;
      S.ioff = L.ioff[sd];
      S.ikey = L.ikey[sd];
      S.imask = L.imask[sd];
    }
  }
  // S1 of every outer quarter of the batch on the device: one launch
  OuterSeg *d_osegs;
  CK(da.get(&d_osegs, 2 * K));
  CK(cp.h2d(d_osegs, osegs.data(), sizeof(OuterSeg) * 2 * K));
  LAUNCH(MSP_K_GRAY, 1, 0, launch_direct_outer(d_osegs, static_cast<int>(2 * K), s));
  InnerSeg *d_segs;
  CK(da.get(&d_segs, 2 * K));
  CK(cp.h2d(d_segs, segs.data(), sizeof(InnerSeg) * 2 * K));
  for (int pass = 0; pass < 2; ++pass) {  // 0: counts, 1: placement
    if (pass == 1) {
      if (M <= (1u << 20)) {
        LAUNCH(MSP_K_BUCKET, 1, 0, launch_direct_inner_offsets(d_segs, static_cast<int>(2 * K), M, s));
      } else {
        uint32_t *scantmp;
        CK(da.get(&scantmp, ((size_t)M + 1 + 4095) / 4096 + 1));
        for (size_t i = 0; i < 2 * K; ++i) {
          LAUNCH(MSP_K_BUCKET, 3, 0, launch_scan_u32(segs[i].cnt, segs[i].ioff, M, scantmp, s));
          CK(cudaMemcpyAsync(segs[i].cnt, segs[i].ioff, sizeof(uint32_t) * M, cudaMemcpyDeviceToDevice, s));
        }
      }
    }
    for (int sd = 0; sd < 2; ++sd) {
      const InnerSeg *sp = d_segs + sd * K;
      LAUNCH(MSP_K_BUCKET, 1, 0, launch_direct_inner_batch(sp, static_cast<int>(K), dp.qi[sd], pass == 1, s));
    }
  }
  return MSP_OK;
}

// The class joins and the verification of the instances `lists` (all of one
// (m, n)), over the residue classes [c_begin, c_end) of each.  Solutions go
// to out[instance] as two words each (unsorted); st (may be null) receives
// passes, records, matches and pairs verified.  With `first`, the matches
// are verified after every launch and the classes stop after the first
// launch that yields a solution (*classes_done: classes joined).  Returns
// MSP_OK, kDirectFallback, or an error status.
int run_direct(const std::vector<DirectLists> &lists, const DirectPlan &dp, uint32_t c_begin, uint32_t c_end,
               DevAlloc &da, Copier &cp, Prof &prof, msp_stats *st, const volatile int *cancel, bool first,
               uint32_t *classes_done, std::vector<std::vector<uint64_t>> &out) {
  cudaStream_t s = cp.s;
  const uint32_t M = 1u << dp.B, cmask = M - 1u;
  const uint32_t K = static_cast<uint32_t>(lists.size());
  out.assign(K, {});
  if (K == 0 || c_begin >= c_end) return MSP_OK;
  std::vector<DirectInst> tab(K);
  std::vector<DirectVerifyInst> vtab(K);
  for (uint32_t k = 0; k < K; ++k) {
    const DirectLists &L = lists[k];
    for (int sd = 0; sd < 2; ++sd) {
      DirectSide &ds = tab[k].side[sd];
      ds.okey = L.d_okey[sd];
      ds.ocls = L.d_ocls[sd];
      ds.ikey = L.ikey[sd];
      ds.ioff = L.ioff[sd];
      ds.no = L.no[sd];
      ds.ni = static_cast<uint32_t>(std::min<uint64_t>(uint64_t(1) << dp.qi[sd], 0xffffffffull));
      DirectVerifyInst &vi = vtab[k];
      vi.side[sd] = ds;
      vi.imask[sd] = L.imask[sd];
      vi.omask[sd] = L.d_omask[sd];
      vi.ovec[sd] = L.d_ovec[sd];
      vi.icol[sd] = L.icol[sd];
    }
    for (int w = 0; w < 4; ++w) vtab[k].dvec[w] = L.dvec[w];
  }
  DirectInst *d_tab;
  DirectVerifyInst *d_vtab;
  CK(da.get(&d_tab, K));
  CK(da.get(&d_vtab, K));
  CK(cp.h2d(d_tab, tab.data(), sizeof(DirectInst) * K));
  CK(cp.h2d(d_vtab, vtab.data(), sizeof(DirectVerifyInst) * K));

  uint32_t *match_key, *match_cls;
  unsigned long long *match_count, *records;
  unsigned int *work, *err;
  CK(da.get(&match_key, kDirectMatchCap));
  CK(da.get(&match_cls, kDirectMatchCap));
  CK(da.get(&match_count, 1));
  CK(da.get(&records, 1));
  CK(da.get(&err, 1));
  CK(cudaMemsetAsync(match_count, 0, sizeof(unsigned long long), s));
  CK(cudaMemsetAsync(records, 0, sizeof(unsigned long long), s));
  CK(cudaMemsetAsync(err, 0, sizeof(unsigned int), s));

  DirectPass p{};
  p.inst = d_tab;
  p.ninst = K;
  p.no[0] = tab[0].side[0].no;
  p.no[1] = tab[0].side[1].no;
  p.class_bits = static_cast<uint32_t>(dp.B);
  p.cmask = cmask;
  p.insert_cap = (5u << dp.TB) / 8;  // about 5 of the 8 slots of a bucket
  p.match_key = match_key;
  p.match_cls = match_cls;
  p.match_count = match_count;
  p.match_cap = kDirectMatchCap;
  p.records = records;
  p.error = err;
  // launches of about 2^32 records (15 ms) and at most 2^20 classes in all:
  // a bounded kernel time, so cancellation (checked between launches) and
  // the kernels of other requests on higher-priority streams get their turn
  const uint32_t ncls = c_end - c_begin;
  const double rec_per_class = std::ldexp(1.0, dp.cols[0] - dp.B) + std::ldexp(1.0, dp.cols[1] - dp.B);
  const uint32_t per_launch = static_cast<uint32_t>(std::max<double>(
      1.0, std::min<double>(std::ldexp(1.0, 32) / rec_per_class, (double)(1u << 20)) / K));
  const uint32_t nlaunch = (ncls + per_launch - 1) / per_launch;
  CK(da.get(&work, nlaunch));
  CK(cudaMemsetAsync(work, 0, sizeof(unsigned int) * nlaunch, s));
  const double per_class_in = 4.0 * (p.no[0] + p.no[1]);

  // ---- verification of the matches [m0, m1) (one block each) ----
  DirectVerify v{};
  v.inst = d_vtab;
  for (int sd = 0; sd < 2; ++sd) {
    v.qi[sd] = dp.qi[sd];
    v.col_o[sd] = dp.col_o[sd];
    v.col_i[sd] = dp.col_i[sd];
  }
  v.W = dp.W;
  v.class_bits = static_cast<uint32_t>(dp.B);
  v.cmask = cmask;
  unsigned long long *cnts;  // solutions, then the pair counters
  unsigned int *ovf;
  CK(da.get(&cnts, 1 + kVerifyPairSlots));
  CK(da.get(&ovf, 1));
  v.sol_count = cnts;
  v.pairs = cnts + 1;
  v.overflow = ovf;
  uint64_t pairs_verified = 0, nsol = 0;
  auto verify = [&](uint64_t m0, uint64_t m1) -> int {
    if (m1 <= m0) return MSP_OK;
    v.match_key = match_key + m0;
    v.match_cls = match_cls + m0;
    uint64_t cap = 1u << 16;
    for (int attempt = 0; attempt < 2; ++attempt) {
      uint64_t *sol;
      CK(da.get(&sol, 3 * cap));
      v.sol = sol;
      v.sol_cap = cap;
      CK(cudaMemsetAsync(cnts, 0, (1 + kVerifyPairSlots) * sizeof(unsigned long long), s));
      CK(cudaMemsetAsync(ovf, 0, sizeof(unsigned int), s));
      NvtxRange nv("msp direct: verification");
      LAUNCH(MSP_K_VERIFY, 1, 0, launch_direct_verify(v, static_cast<unsigned>(m1 - m0), s));
      unsigned long long hcs[1 + kVerifyPairSlots];
      unsigned int ovf_h = 0;
      CK(cp.d2h(hcs, cnts, sizeof(hcs)));
      CK(cp.d2h(&ovf_h, ovf, sizeof(ovf_h)));
      CK(cudaStreamSynchronize(s));
      if (ovf_h) return kDirectFallback;
      unsigned long long hc[2] = {hcs[0], 0};
      for (int k = 1; k <= kVerifyPairSlots; ++k) hc[1] += hcs[k];
      if (hc[0] <= cap) {
        pairs_verified += hc[1];
        nsol += hc[0];
        std::vector<uint64_t> h(3 * hc[0]);
        if (hc[0]) {
          CK(cp.d2h(h.data(), sol, sizeof(uint64_t) * 3 * hc[0]));
          CK(cudaStreamSynchronize(s));
        }
        da.free1(sol, sizeof(uint64_t) * 3 * cap);
        for (uint64_t i = 0; i < hc[0]; ++i) {
          const uint64_t k = h[3 * i + 2];
          if (k >= K) return fail(MSP_ECUDA, "verification produced an invalid instance tag");
          out[k].push_back(h[3 * i]);
          out[k].push_back(h[3 * i + 1]);
        }
        return MSP_OK;
      }
      da.free1(sol, sizeof(uint64_t) * 3 * cap);
      if (hc[0] > (1ull << 28)) return fail(MSP_EOVERFLOW, "more than 2^28 solutions");
      cap = hc[0];
    }
    return MSP_OK;
  };

  int passes = 0;
  uint64_t verified_to = 0;  // first-solution mode: matches verified so far
  uint32_t classes_run = 0;
  // A cancelable solve (serving loop) keeps at most kInFlight join launches
  // queued, so that a cancellation seen before a launch stops the solve
  // within a few launches; other solves queue every launch at once.
  constexpr uint32_t kInFlight = 2;
  EventRing ring(cancel ? kInFlight : 0);
  CK(ring.status);
  for (uint32_t li = 0; li < nlaunch; ++li) {
    if (cancel) {
      if (li >= kInFlight) CK(ring.wait(li % kInFlight));
      if (*cancel) return fail(MSP_ECANCELED, "request canceled");
    }
    p.c0 = c_begin + li * per_launch;
    p.nclass = std::min(per_launch, c_end - p.c0);
    p.work = work + li;
    // algorithmic bytes: 4 per record (its inner key) plus one bucket offset
    // per outer subset and class; the exact record count replaces this
    // estimate once the solve ends
    const double rec_est = (double)K * p.nclass * rec_per_class;
    LAUNCH(MSP_K_DIRECT, 1, static_cast<uint64_t>(4.0 * rec_est + per_class_in * p.nclass * K),
           launch_direct_join(dp.TB, p, s));
    if (cancel) CK(ring.record(li % kInFlight, s));
    ++passes;
    classes_run += p.nclass;
    if (first) {
      // stop after the launch whose matches verify to a solution
      unsigned long long nm = 0;
      CK(cp.d2h(&nm, match_count, sizeof(nm)));
      CK(cudaStreamSynchronize(s));
      if (nm > kDirectMatchCap) break;
      if (nm > verified_to) {
        const int rc = verify(verified_to, nm);
        if (rc != MSP_OK) return rc;
        verified_to = nm;
        if (nsol) break;
      }
    }
  }
  if (classes_done) *classes_done = classes_run;
  unsigned long long nmatch = 0, nrec = 0;
  unsigned int err_h = 0;
  CK(cp.d2h(&nmatch, match_count, sizeof(nmatch)));
  CK(cp.d2h(&nrec, records, sizeof(nrec)));
  CK(cp.d2h(&err_h, err, sizeof(err_h)));
  CK(cudaStreamSynchronize(s));
  prof.flush();
  if (st) {
    st->passes = passes;
    st->records_done = nrec;
    st->key_matches = nmatch;
    if (prof.on) st->kernel_bytes[MSP_K_DIRECT] = 4 * nrec + static_cast<uint64_t>(per_class_in * ncls * K);
  }
  if (err_h || nmatch > kDirectMatchCap) return kDirectFallback;
  if (!first || nsol == 0) {
    const int rc = verify(verified_to, nmatch);
    if (rc != MSP_OK) return rc;
  }
  if (st) st->pairs_verified = pairs_verified;
  return MSP_OK;
}

}  // namespace

// Solves `inst` on the direct pass.  Returns MSP_OK with res (unsorted
// two-word masks), kDirectFallback when another path must solve it (out of
// memory for the inner lists, a class beyond the kernel's bounds, a match
// list or candidate list overflow), or an error status.
int solve_direct(msp_instance *inst, const DirectPlan &dp, const Plan &kp, size_t budget, Prof &prof,
                 std::vector<uint64_t> &res) {
  const int n = inst->n;
  msp_stats &st = inst->stats;
  cudaStream_t s = inst->stream;
  const uint32_t M = 1u << dp.B;
  if (direct_footprint(dp) > budget) return kDirectFallback;
  if (inst->part >= inst->parts) return fail(MSP_EINVAL, "class part must be below the number of parts");

  st.quarter[0] = dp.qo[0];
  st.quarter[1] = dp.qo[1];
  st.quarter[2] = dp.qi[0];
  st.quarter[3] = dp.qi[1];
  st.class_bits = dp.B;
  st.class_rows = dp.t;
  st.digit_bits = 0;

  DevAlloc da(s);
  Copier cp{&st, s};
  std::vector<DirectLists> lists(1);
  {
    NvtxRange nv("msp direct: quarter lists");
    uint32_t *cnt, *scantmp;
    CK(da.get(&cnt, (size_t)M + 1));
    CK(da.get(&scantmp, ((size_t)M + 1 + 4095) / 4096 + 1));
    const int rc = build_direct_lists(inst->A.data(), inst->d.data(), inst->m, n, dp, kp, da, cp, prof, cnt,
                                      scantmp, lists[0]);
    if (rc != MSP_OK) return rc;
    da.free1(cnt, sizeof(uint32_t) * ((size_t)M + 1));
  }

  // ---- C1: row-1 candidate pairs (the metric's unit of work) ----
  {
    int32_t *d_a1;
    ulonglong2 *d_dp;  // 128-bit counters
    unsigned long long *d_c1;
    const int d1 = inst->d[0];
    CK(da.get(&d_a1, n));
    CK(da.get(&d_dp, 2 * ((size_t)d1 + 1)));
    CK(da.get(&d_c1, 2));
    CK(cp.h2d(d_a1, inst->A.data(), sizeof(int32_t) * n));
    LAUNCH(MSP_K_C1, 1, 0, launch_c1_dp(d_a1, n, d1, d_dp, d_c1, s));
    unsigned long long c1h[2];
    CK(cp.d2h(c1h, d_c1, sizeof(c1h)));
    CK(cudaStreamSynchronize(s));
    st.row1_candidates_lo = c1h[0];
    st.row1_candidates_hi = c1h[1];
  }

  const uint32_t c_begin = static_cast<uint32_t>((uint64_t)M * inst->part / inst->parts);
  const uint32_t c_end = static_cast<uint32_t>((uint64_t)M * (inst->part + 1) / inst->parts);
  st.classes_total = M;
  st.classes_done = c_end - c_begin;
  std::vector<std::vector<uint64_t>> out;
  uint32_t done = 0;
  NvtxRange nv("msp direct: class joins and verification");
  const int rc =
      run_direct(lists, dp, c_begin, c_end, da, cp, prof, &st, inst->cancel, inst->first_only, &done, out);
  st.classes_done = done;
  if (rc != MSP_OK) return rc;
  res = std::move(out[0]);
  st.device_bytes = da.peak;
  da.release();
  CK(cudaStreamSynchronize(s));
  prof.flush();
  return MSP_OK;
}

// msp_solve_batch on the direct pass: every instance's lists, then one join
// launch (per 2^20 classes) over the classes of all instances and one
// verification launch over all matches.  raw[k]: unsorted two-word masks of
// instance k.  Returns MSP_OK, kDirectFallback or an error status.
int solve_batch_direct(const int32_t *const *A, const int32_t *const *d, int m, int n, int count,
                       std::vector<std::vector<uint64_t>> &raw, cudaStream_t s, size_t budget) {
  raw.assign(count, {});
  const DirectPlan dp = make_direct_plan(m, n, -1);
  if (!dp.ok) return kDirectFallback;
  const Plan kp = make_plan(m, n);
  const uint32_t M = 1u << dp.B;
  // feasible right-hand sides only
  std::vector<int> idx;
  for (int k = 0; k < count; ++k) {
    bool feasible = true;
    for (int i = 0; i < m && feasible; ++i) {
      int64_t rs = 0;
      for (int j = 0; j < n; ++j) rs += A[k][(size_t)i * n + j];
      feasible = d[k][i] <= rs;
    }
    if (feasible) idx.push_back(k);
  }
  const uint32_t K = static_cast<uint32_t>(idx.size());
  if (K == 0) return MSP_OK;
  // tags instance << B | class must fit 32 bits; lists of all instances
  // must fit the budget
  if ((uint64_t)K << dp.B > (1ull << 32)) return kDirectFallback;
  const double per_inst = 8.0 * (std::ldexp(1.0, dp.qi[0]) + std::ldexp(1.0, dp.qi[1])) +
                          16.0 * (std::ldexp(1.0, dp.B) + 1) + (64 << 10);
  if (per_inst * K + (double)direct_footprint(dp) > (double)budget) return kDirectFallback;

  DevAlloc da(s);
  Copier cp{nullptr, s};
  msp_stats scratch{};
  Prof prof;
  prof.s = s;
  prof.st = &scratch;
  std::vector<DirectLists> lists;
  {
    const int rc = build_direct_lists_batch(A, d, idx, m, n, dp, kp, da, cp, prof, lists);
    if (rc != MSP_OK) return rc;
  }
  std::vector<std::vector<uint64_t>> out;
  const int rc = run_direct(lists, dp, 0, M, da, cp, prof, nullptr, nullptr, false, nullptr, out);
  if (rc != MSP_OK) return rc;
  for (uint32_t k = 0; k < K; ++k) raw[idx[k]] = std::move(out[k]);
  da.release();
  CK(cudaStreamSynchronize(s));
  return MSP_OK;
}

}  // namespace msp
