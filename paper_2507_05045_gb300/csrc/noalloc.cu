// msp_solve_small_noalloc: an exhaustive solve of a small instance that
// allocates no device memory.
//
// Some callers cannot allocate device memory at solve time: a process whose
// device memory is owned by another framework's allocator (and may be fully
// reserved by it), a serving loop that must not risk an out-of-memory
// failure or an allocator stall in the middle of a request, or code running
// under a fixed device-memory quota set at start-up.  For them this entry
// point runs the exact two-phase residue pass of msp_solve_all (the same
// kernels) with every intermediate buffer - quarter lists, class buckets,
// partition counters and offsets, the half-pair records, matched keys,
// recovered candidates and solutions - carved out of one file-scope static
// device array of kNoallocScratchBytes.  Every device that loads the library
// holds that array until the process exits.
//
// Set-up: every call resolves the array's device address on the caller's
// current device with cudaGetSymbolAddress (a cheap lookup), so the address
// stays right after a device reset reloads the module.  A call synchronises
// its stream (it reads match, candidate and solution counts back to the host
// between phases), so it must not be made while that stream is capturing a
// CUDA graph.  All calls share the one array and it keeps the last call's
// contents, so the counters that must start at zero are cleared on every
// call, and two calls that overlap on the GPU (different streams or threads
// without ordering) race on it: serialise them.
#include "host_internal.h"

#include <algorithm>
#include <cstring>

namespace {

// 24 MiB: 2^20 eight-byte records per side (n <= 40) plus lists and tables.
constexpr size_t kNoallocScratchBytes = size_t(24) << 20;
constexpr int kNoallocMaxN = 40;
constexpr uint64_t kNoallocMatchCap = 1u << 13;
constexpr uint64_t kNoallocCandCap = 1u << 17;
constexpr uint64_t kNoallocSolCap = 1u << 17;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Device address of the scratch array on the current device, looked up on
// every call.
int scratch_address(unsigned char **out) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    return msp::fail(MSP_ECUDA, std::string("cudaGetSymbolAddress of the scratch array: ") + cudaGetErrorString(e));
  *out = static_cast<unsigned char *>(p);
  return MSP_OK;
}

// Bump allocation inside the scratch array (256-byte aligned pieces).
struct Carve {
  unsigned char *base;
  size_t used = 0;
  bool ok = true;
  template <typename T>
  T *take(size_t count) {
    const size_t bytes = ((std::max<size_t>(count, 1) * sizeof(T)) + 255) & ~size_t(255);
    if (used + bytes > kNoallocScratchBytes) {
      ok = false;
      return nullptr;
    }
    T *p = reinterpret_cast<T *>(base + used);
    used += bytes;
    return p;
  }
};

#define NA_CK(call)                                                                         \
  do {                                                                                      \
    const cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) return msp::fail(MSP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

using namespace msp;

extern "C" int msp_solve_small_noalloc(const int32_t *A, const int32_t *d, int m, int n, uint64_t *masks,
                                       size_t cap, size_t *count, void *stream) {
  if (!count) return fail(MSP_EINVAL, "count must be non-null");
  *count = 0;
  if (cap && !masks) return fail(MSP_EINVAL, "masks must be non-null when cap > 0");
  int rc = validate(A, d, m, n);
  if (rc != MSP_OK) return rc;
  if (n > kNoallocMaxN)
    return fail(MSP_ERANGE, "msp_solve_small_noalloc: n above 40 (its static scratch holds at most 2^20 "
                            "half-pair records per side); use msp_solve_all");
  unsigned char *scratch = nullptr;
  rc = scratch_address(&scratch);
  if (rc != MSP_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  const Plan p = make_plan(m, n);  // n <= 40: one residue class (B = 0)
  for (int i = 0; i < m; ++i) {
    int64_t rs = 0;
    for (int j = 0; j < n; ++j) rs += A[(size_t)i * n + j];
    if (d[i] > rs) return MSP_OK;  // no solution
  }
  if (p.B != 0) return fail(MSP_ERANGE, "msp_solve_small_noalloc: instance needs more than one class");

  // ---- constants and packed columns (as msp_solve_all) ----
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
  uint64_t pcol[kNoallocMaxN * kMaxVecWords] = {};
  uint64_t kcol[kNoallocMaxN];
  uint32_t ccol[kNoallocMaxN];
  int64_t col[kMaxRows];
  for (int j = 0; j < n; ++j) {
    uint32_t c = 0;
    for (int i = 0; i < m; ++i) {
      col[i] = A[(size_t)i * n + j];
      pcol[j * kMaxVecWords + i / 4] |= static_cast<uint64_t>(col[i]) << (16 * (i % 4));
    }
    kcol[j] = key_of(p, col);
    for (int i = 0; i < p.t; ++i) c += p.c_row[i] * static_cast<uint32_t>(col[i]);
    ccol[j] = c;
  }
  int64_t dv[kMaxRows];
  for (int i = 0; i < m; ++i) {
    dv[i] = d[i];
    ic.dvec[i / 4] |= static_cast<uint64_t>(dv[i]) << (16 * (i % 4));
  }
  ic.kd = key_of(p, dv);
  ic.cd = class_of(p, dv);
  const uint32_t M = 1u, cmask = 0u;
  const int nd = 1 << p.Dx;

  // ---- carve every buffer out of the static scratch ----
  Carve cv{scratch};
  uint64_t *d_pcol = cv.take<uint64_t>(kNoallocMaxN * kMaxVecWords);
  uint64_t *d_kcol = cv.take<uint64_t>(kNoallocMaxN);
  uint32_t *d_ccol = cv.take<uint32_t>(kNoallocMaxN);
  QuarterDev qd[4];
  for (int k = 0; k < 4; ++k) {
    qd[k].q = p.q[k];
    qd[k].size = int64_t(1) << p.q[k];
    qd[k].vec = cv.take<uint64_t>((size_t)p.W * qd[k].size);
    qd[k].key = cv.take<uint64_t>(qd[k].size);
    qd[k].cls = cv.take<uint32_t>(qd[k].size);
    qd[k].v1 = cv.take<uint32_t>(qd[k].size);
  }
  BucketDev bd[4];
  const int qk[4] = {0, 2, 1, 3};
  for (int l = 0; l < 4; ++l) {
    bd[l].size = qd[qk[l]].size;
    bd[l].key = cv.take<uint64_t>(bd[l].size);
    bd[l].cls = cv.take<uint32_t>(bd[l].size);
    bd[l].idx = cv.take<uint32_t>(bd[l].size);
    bd[l].off = cv.take<uint32_t>(M + 1);
  }
  uint32_t *d_hist = cv.take<uint32_t>(M);
  uint32_t *d_cursor = cv.take<uint32_t>(M + 1);
  uint32_t *d_scantmp = cv.take<uint32_t>(4);
  PassDev pd{};
  pd.cmask = cmask;
  pd.D = p.Dx;
  pd.S = p.S;
  for (int side = 0; side < 2; ++side) {
    const BucketDev &o = bd[side == 0 ? 0 : 2];
    const BucketDev &in = bd[side == 0 ? 1 : 3];
    SideGen &g = pd.side[side];
    g.okey = o.key;
    g.ocls = o.cls;
    g.osize = o.size;
    g.ikey = in.key;
    g.isize = in.size;
    g.ioff = in.off;
    const int64_t per_bucket = std::max<int64_t>(1, in.size / M);
    g.slice_outer = std::max<int64_t>(1, (int64_t(1) << 19) / per_bucket);
    g.slices = static_cast<int>((o.size + g.slice_outer - 1) / g.slice_outer);
    pd.cnt[side] = cv.take<uint32_t>((size_t)g.slices * nd);
    pd.segstart[side] = cv.take<uint64_t>(nd);
    pd.seglen[side] = cv.take<uint32_t>(nd);
    pd.classtot[side] = cv.take<uint64_t>(1);
    pd.classbase[side] = cv.take<uint64_t>(1);
    pd.rec[side] = cv.take<uint64_t>(size_t(1) << (side == 0 ? p.lgL : p.lgR));
  }
  pd.match_cap = kNoallocMatchCap;
  pd.match_key = cv.take<uint64_t>(kNoallocMatchCap);
  pd.match_cls = cv.take<uint32_t>(kNoallocMatchCap);
  pd.match_count = cv.take<unsigned long long>(1);
  pd.big_cap = static_cast<uint32_t>(nd);
  pd.big_list = cv.take<uint32_t>(nd);
  pd.big_count = cv.take<unsigned int>(1);
  RecoverDev rd{};
  for (int side = 0; side < 2; ++side) {
    rd.cand_count[side] = cv.take<unsigned long long>(kNoallocMatchCap);
    rd.cand_off[side] = cv.take<unsigned long long>(kNoallocMatchCap + 1);
    rd.cand_cur[side] = cv.take<unsigned long long>(kNoallocMatchCap);
    rd.cand[side] = cv.take<uint64_t>(kNoallocCandCap);
  }
  rd.cand_match[0] = cv.take<uint32_t>(kNoallocCandCap);
  unsigned long long *tmp64 = cv.take<unsigned long long>(4);
  uint64_t *sol = cv.take<uint64_t>(2 * kNoallocSolCap);
  unsigned long long *cnts = cv.take<unsigned long long>(2);
  if (!cv.ok) return fail(MSP_ERANGE, "msp_solve_small_noalloc: instance does not fit the static scratch");

  // ---- S0 .. S2: columns, Gray-code quarter lists, class buckets ----
  NA_CK(cudaMemcpyAsync(d_pcol, pcol, sizeof(pcol), cudaMemcpyHostToDevice, s));
  NA_CK(cudaMemcpyAsync(d_kcol, kcol, sizeof(uint64_t) * n, cudaMemcpyHostToDevice, s));
  NA_CK(cudaMemcpyAsync(d_ccol, ccol, sizeof(uint32_t) * n, cudaMemcpyHostToDevice, s));
  for (int k = 0; k < 4; ++k) NA_CK(launch_gray(ic, d_pcol, d_kcol, d_ccol, qd[k], p.col0[k], s));
  const int64_t mul[4] = {1, 1, -1, -1};
  const uint64_t kadd[4] = {0, 0, ic.kd, 0};
  const uint32_t cadd[4] = {0, 0, ic.cd, 0};
  for (int l = 0; l < 4; ++l) {
    const QuarterDev &q = qd[qk[l]];
    NA_CK(cudaMemsetAsync(d_hist, 0, sizeof(uint32_t) * M, s));
    NA_CK(launch_count_classes(q.cls, q.size, static_cast<uint32_t>(mul[l]), cadd[l], cmask, d_hist, s));
    NA_CK(launch_scan_u32(d_hist, bd[l].off, M, d_scantmp, s));
    NA_CK(cudaMemcpyAsync(d_cursor, bd[l].off, sizeof(uint32_t) * M, cudaMemcpyDeviceToDevice, s));
    NA_CK(launch_bucket_scatter(q, mul[l], kadd[l], cadd[l], cmask, d_cursor, bd[l], s));
  }

  // ---- S3 .. S5: the single residue pass, exact two-phase form ----
  NA_CK(cudaMemsetAsync(pd.match_count, 0, sizeof(unsigned long long), s));
  pd.c0 = 0;
  pd.nclass = 1;
  NA_CK(launch_gen_count(pd, s));
  NA_CK(launch_counts_to_offsets(pd, s));
  NA_CK(cudaMemsetAsync(pd.classbase[0], 0, sizeof(uint64_t), s));
  NA_CK(cudaMemsetAsync(pd.classbase[1], 0, sizeof(uint64_t), s));
  NA_CK(launch_gen_scatter(pd, 1, s));
  NA_CK(cudaMemsetAsync(pd.big_count, 0, sizeof(unsigned int), s));
  NA_CK(launch_join(pd, 1, s));
  NA_CK(launch_join_big(pd, 1, s));
  unsigned long long nmatch = 0;
  NA_CK(cudaMemcpyAsync(&nmatch, pd.match_count, sizeof(nmatch), cudaMemcpyDeviceToHost, s));
  NA_CK(cudaStreamSynchronize(s));
  if (nmatch > kNoallocMatchCap)
    return fail(MSP_EOVERFLOW, "msp_solve_small_noalloc: more matched keys than its scratch holds (8192)");
  if (nmatch == 0) return MSP_OK;

  // ---- S6: recovery and exact verification ----
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
  for (int side = 0; side < 2; ++side) {
    NA_CK(cudaMemsetAsync(rd.cand_count[side], 0, sizeof(unsigned long long) * nmatch, s));
    NA_CK(cudaMemsetAsync(rd.cand_cur[side], 0, sizeof(unsigned long long) * nmatch, s));
  }
  NA_CK(launch_recover(rd, false, s));
  unsigned long long ncand[2];
  for (int side = 0; side < 2; ++side) {
    NA_CK(launch_scan_u64(rd.cand_count[side], rd.cand_off[side], nmatch, tmp64, s));
    NA_CK(cudaMemcpyAsync(&ncand[side], rd.cand_off[side] + nmatch, sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, s));
  }
  NA_CK(cudaStreamSynchronize(s));
  if (ncand[0] > kNoallocCandCap || ncand[1] > kNoallocCandCap)
    return fail(MSP_EOVERFLOW, "msp_solve_small_noalloc: more candidates than its scratch holds (131072)");
  rd.cand_cap[0] = ncand[0];
  rd.cand_cap[1] = ncand[1];
  NA_CK(launch_recover(rd, true, s));
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
  vd.sol = sol;
  vd.sol_cap = kNoallocSolCap;
  vd.sol_count = cnts;
  vd.pairs_checked = cnts + 1;
  NA_CK(cudaMemsetAsync(cnts, 0, 2 * sizeof(unsigned long long), s));
  NA_CK(launch_verify(vd, s));
  unsigned long long nsol = 0;
  NA_CK(cudaMemcpyAsync(&nsol, cnts, sizeof(nsol), cudaMemcpyDeviceToHost, s));
  NA_CK(cudaStreamSynchronize(s));
  if (nsol > kNoallocSolCap)
    return fail(MSP_EOVERFLOW, "msp_solve_small_noalloc: more solutions than its scratch holds (131072)");

  // ---- S7: low words (n <= 40 fits one word) into the caller's buffer,
  //      sorted and de-duplicated in place ----
  const size_t ncopy = std::min<size_t>(nsol, cap);
  if (ncopy) {
    NA_CK(cudaMemcpy2DAsync(masks, sizeof(uint64_t), sol, 2 * sizeof(uint64_t), sizeof(uint64_t), ncopy,
                            cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
  }
  if (nsol > cap) {
    *count = nsol;  // upper bound (duplicates not removed): retry with a larger buffer
    return fail(MSP_EOVERFLOW, "masks buffer smaller than the number of solutions (count holds the need)");
  }
  std::sort(masks, masks + ncopy);
  *count = static_cast<size_t>(std::unique(masks, masks + ncopy) - masks);
  return MSP_OK;
}
