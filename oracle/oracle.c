/*
 * CPU oracle for the feasibility market split problem (n-SSP).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header, table or
 * helper with the CUDA path.
 *
 * What it computes (Section 1, eq. 1): for A in N0^{m x n} and d in N0^m,
 *     Sol(A, d) = { x in {0,1}^n : sum_j a_ij x_j = d_i for every row i },
 * every solution, as bitmasks (bit j of little-endian 64-bit word j/64 is
 * x_j), sorted ascending as unsigned integers (most significant word first).
 *
 * Functions:
 *   msp_oracle_brute   - the definition written out: every x in binary order.
 *   msp_oracle_mitm    - Horowitz-Sahni two-list meet in the middle (cited in
 *                        Section 2) on full m-row vectors, split at n/2,
 *                        sliced by the residue of the exact row-1 value so a
 *                        slice fits in memory.
 *   msp_oracle_subset_count - textbook subset-sum counting DP (number of
 *                        subsets of given weights with a given sum); with the
 *                        row-1 weights and d_1 it is the number of row-1
 *                        candidates of Algorithm 2 (all pairs of a left and a
 *                        right half whose row-1 sums add to d_1).
 *   msp_oracle_residue_hist - DP histogram of subsets of a column set by the
 *                        tuple of row residues (rows 1..t modulo M_1..M_t);
 *                        the residue-class sizes of a partition of the row-1
 *                        (and further rows') key space.
 */
#define _GNU_SOURCE
#include "oracle.h"

#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXW 2 /* mask words: n <= 128 */

static int words_for(int n) { return (n + 63) / 64; }

static void set_bit(uint64_t *mask, int j) { mask[j >> 6] |= (uint64_t)1 << (j & 63); }

/* ---- sorting of the output masks (most significant word first) ---- */
static int g_sort_words;
static int cmp_mask(const void *pa, const void *pb) {
  const uint64_t *a = (const uint64_t *)pa, *b = (const uint64_t *)pb;
  for (int w = g_sort_words - 1; w >= 0; --w) {
    if (a[w] < b[w]) return -1;
    if (a[w] > b[w]) return 1;
  }
  return 0;
}
static void sort_masks(uint64_t *out, int64_t count, int words) {
  g_sort_words = words;
  qsort(out, (size_t)count, sizeof(uint64_t) * (size_t)words, cmp_mask);
}

int msp_oracle_words(int n) { return words_for(n); }

/* ------------------------------------------------------------------ */
/* Brute force: the definition of Sol(A, d) written out (eq. 1).       */
/* ------------------------------------------------------------------ */
int64_t msp_oracle_brute(const int32_t *A, const int32_t *d, int m, int n,
                         uint64_t *out, int64_t cap) {
  if (m < 1 || n < 1 || n > 40) return -1;
  const int words = words_for(n);
  int64_t count = 0;
  const uint64_t total = (uint64_t)1 << n;
  for (uint64_t x = 0; x < total; ++x) {
    int ok = 1;
    for (int i = 0; i < m && ok; ++i) {
      int64_t s = 0;
      for (int j = 0; j < n; ++j)
        if ((x >> j) & 1) s += A[(size_t)i * n + j];
      ok = (s == d[i]);
    }
    if (!ok) continue;
    if (count < cap) {
      uint64_t *dst = out + (size_t)count * words;
      memset(dst, 0, sizeof(uint64_t) * words);
      dst[0] = x;
    }
    ++count;
  }
  if (count <= cap) sort_masks(out, count, words);
  return count;
}

/* ------------------------------------------------------------------ */
/* Meet in the middle (Horowitz-Sahni two lists, Section 2).           */
/* ------------------------------------------------------------------ */
typedef struct {
  int m;
  const int32_t *vec; /* [count][m] */
} vec_ctx;

static int cmp_vec_idx(const void *pa, const void *pb, void *vctx) {
  const vec_ctx *c = (const vec_ctx *)vctx;
  const int32_t *a = c->vec + (size_t)(*(const int64_t *)pa) * c->m;
  const int32_t *b = c->vec + (size_t)(*(const int64_t *)pb) * c->m;
  for (int i = 0; i < c->m; ++i) {
    if (a[i] < b[i]) return -1;
    if (a[i] > b[i]) return 1;
  }
  return 0;
}

/* Compare stored vector idx with target t; <0, 0, >0 like memcmp. */
static int cmp_to_target(const vec_ctx *c, int64_t idx, const int32_t *t) {
  const int32_t *a = c->vec + (size_t)idx * c->m;
  for (int i = 0; i < c->m; ++i) {
    if (a[i] < t[i]) return -1;
    if (a[i] > t[i]) return 1;
  }
  return 0;
}

/*
 * Enumerate all subsets of the columns [c0, c0 + k) in binary-counter order.
 * Going from u-1 to u clears bits 0..z-1 and sets bit z (z = ctz(u)), so
 * v(u) = v(u-1) + col_z - (col_0 + ... + col_{z-1}).  Calls visit(u, v).
 */
typedef struct {
  const int32_t *A;
  int m, n, c0, k;
  int32_t *col;  /* [k][m] columns */
  int32_t *pre;  /* [k][m] prefix sums of columns */
} half_t;

static void half_init(half_t *h, const int32_t *A, int m, int n, int c0, int k) {
  h->A = A; h->m = m; h->n = n; h->c0 = c0; h->k = k;
  h->col = (int32_t *)calloc((size_t)(k > 0 ? k : 1) * m, sizeof(int32_t));
  h->pre = (int32_t *)calloc((size_t)(k > 0 ? k : 1) * m, sizeof(int32_t));
  for (int z = 0; z < k; ++z)
    for (int i = 0; i < m; ++i) {
      h->col[(size_t)z * m + i] = A[(size_t)i * n + c0 + z];
      h->pre[(size_t)z * m + i] = (z > 0 ? h->pre[(size_t)(z - 1) * m + i] + h->col[(size_t)(z - 1) * m + i] : 0);
    }
}
static void half_free(half_t *h) { free(h->col); free(h->pre); }
static inline void half_step(const half_t *h, uint64_t u, int32_t *v) {
  if (u == 0) { memset(v, 0, sizeof(int32_t) * h->m); return; }
  const int z = __builtin_ctzll(u);
  for (int i = 0; i < h->m; ++i) v[i] += h->col[(size_t)z * h->m + i] - h->pre[(size_t)z * h->m + i];
}

typedef struct {
  uint64_t *buf; /* [cnt][words] */
  int64_t cnt, capacity;
} mask_list;

static int mask_list_push(mask_list *l, const uint64_t *mask, int words) {
  if (l->cnt == l->capacity) {
    int64_t nc = l->capacity ? 2 * l->capacity : 64;
    uint64_t *nb = (uint64_t *)realloc(l->buf, sizeof(uint64_t) * (size_t)words * (size_t)nc);
    if (!nb) return -1;
    l->buf = nb;
    l->capacity = nc;
  }
  memcpy(l->buf + (size_t)l->cnt * words, mask, sizeof(uint64_t) * words);
  ++l->cnt;
  return 0;
}

int64_t msp_oracle_mitm(const int32_t *A, const int32_t *d, int m, int n,
                        int slices, uint64_t *out, int64_t cap) {
  if (m < 1 || m > 64 || n < 1 || n > 80) return -1;
  for (int i = 0; i < m; ++i)
    if (d[i] < 0) return 0;
  const int words = words_for(n);
  const int nl = n / 2, nr = n - nl;
  if (slices < 1) slices = 1;
  half_t HL, HR;
  half_init(&HL, A, m, n, 0, nl);
  half_init(&HR, A, m, n, nl, nr);
  int64_t count = 0;
  int failed = 0;

#pragma omp parallel for schedule(dynamic, 1)
  for (int p = 0; p < slices; ++p) {
    int bad;
#pragma omp atomic read
    bad = failed;
    if (bad) continue;
    /* Left subsets u whose exact row-1 value is congruent to p mod slices. */
    const uint64_t nleft = (uint64_t)1 << nl;
    int32_t v[64];
    uint64_t sz = 0;
    for (uint64_t u = 0; u < nleft; ++u) {
      half_step(&HL, u, v);
      if (v[0] % slices == p) ++sz;
    }
    int32_t *vec = (int32_t *)malloc(sizeof(int32_t) * (size_t)m * (sz ? sz : 1));
    uint64_t *um = (uint64_t *)malloc(sizeof(uint64_t) * (sz ? sz : 1));
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (sz ? sz : 1));
    mask_list found = {0, 0, 0};
    if (!vec || !um || !idx) {
#pragma omp atomic write
      failed = 1;
      free(vec); free(um); free(idx);
      continue;
    }
    uint64_t c = 0;
    for (uint64_t u = 0; u < nleft; ++u) {
      half_step(&HL, u, v);
      if (v[0] % slices != p) continue;
      memcpy(vec + (size_t)c * m, v, sizeof(int32_t) * m);
      um[c] = u;
      idx[c] = (int64_t)c;
      ++c;
    }
    vec_ctx ctx = {m, vec};
    qsort_r(idx, sz, sizeof(int64_t), cmp_vec_idx, &ctx);

    /* Right subsets w: every left vector equal to the target d - v(w). */
    const uint64_t nright = (uint64_t)1 << nr;
    int32_t t[64];
    uint64_t mask[MAXW];
    for (uint64_t w = 0; w < nright; ++w) {
      half_step(&HR, w, v);
      int neg = 0;
      for (int i = 0; i < m; ++i) {
        t[i] = d[i] - v[i];
        if (t[i] < 0) neg = 1;
      }
      if (neg || t[0] % slices != p) continue;
      int64_t lo = 0, hi = (int64_t)sz; /* first stored vector >= t */
      while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (cmp_to_target(&ctx, idx[mid], t) < 0) lo = mid + 1; else hi = mid;
      }
      for (int64_t q = lo; q < (int64_t)sz && cmp_to_target(&ctx, idx[q], t) == 0; ++q) {
        memset(mask, 0, sizeof(mask));
        const uint64_t u = um[idx[q]];
        for (int j = 0; j < nl; ++j)
          if ((u >> j) & 1) set_bit(mask, j);
        for (int j = 0; j < nr; ++j)
          if ((w >> j) & 1) set_bit(mask, nl + j);
        if (mask_list_push(&found, mask, words) != 0) {
#pragma omp atomic write
          failed = 1;
          break;
        }
      }
    }
    free(vec); free(um); free(idx);
#pragma omp critical(msp_oracle_out)
    {
      for (int64_t q = 0; q < found.cnt; ++q) {
        if (count < cap)
          memcpy(out + (size_t)count * words, found.buf + (size_t)q * words, sizeof(uint64_t) * words);
        ++count;
      }
    }
    free(found.buf);
  }
  half_free(&HL);
  half_free(&HR);
  if (failed) return -2;
  if (count <= cap) sort_masks(out, count, words);
  return count;
}

/* ------------------------------------------------------------------ */
/* Subset-sum counting DP (128-bit counts).                            */
/* ------------------------------------------------------------------ */
int msp_oracle_subset_count(const int32_t *w, int n, int64_t target, uint64_t out[2]) {
  out[0] = out[1] = 0;
  if (n < 0 || n > 127) return -1;
  int64_t total = 0;
  for (int j = 0; j < n; ++j) {
    if (w[j] < 0) return -1;
    total += w[j];
  }
  if (target < 0 || target > total) return 0;
  unsigned __int128 *cnt = (unsigned __int128 *)calloc((size_t)total + 1, sizeof(unsigned __int128));
  if (!cnt) return -2;
  cnt[0] = 1;
  int64_t reach = 0;
  for (int j = 0; j < n; ++j) {
    /* Either column j is out (count stays) or in (shift by w_j). */
    for (int64_t s = reach; s >= 0; --s) cnt[s + w[j]] += cnt[s];
    /* (w_j = 0 doubles every count: each subset may or may not hold j.) */
    reach += w[j];
  }
  out[0] = (uint64_t)cnt[target];
  out[1] = (uint64_t)(cnt[target] >> 64);
  free(cnt);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Residue-class histogram DP.                                         */
/* ------------------------------------------------------------------ */
/*
 * For the columns cols[0..ncols) count the subsets S by their residue tuple
 * (sum_{j in S} a_ij mod mods[i]) for rows i = 0..t-1.  The tuple is stored
 * at index r_0 + mods[0] * (r_1 + mods[1] * (r_2 + ...)) (row 1 varies
 * fastest).  out must hold prod(mods) entries.  Counts are exact while they
 * fit 64 bits (ncols <= 63).
 */
int msp_oracle_residue_hist(const int32_t *A, int m, int n, const int32_t *cols, int ncols,
                            int t, const int32_t *mods, uint64_t *out) {
  if (t < 1 || t > m || ncols < 0 || ncols > 63) return -1;
  int64_t states = 1;
  for (int i = 0; i < t; ++i) {
    if (mods[i] < 1) return -1;
    states *= mods[i];
    if (states > ((int64_t)1 << 26)) return -1;
  }
  uint64_t *cur = (uint64_t *)calloc((size_t)states, sizeof(uint64_t));
  uint64_t *nxt = (uint64_t *)calloc((size_t)states, sizeof(uint64_t));
  if (!cur || !nxt) { free(cur); free(nxt); return -2; }
  cur[0] = 1;
  int32_t r[64];
  for (int c = 0; c < ncols; ++c) {
    const int j = cols[c];
    if (j < 0 || j >= n) { free(cur); free(nxt); return -1; }
    memcpy(nxt, cur, sizeof(uint64_t) * (size_t)states); /* column j left out */
    for (int64_t s = 0; s < states; ++s) {
      if (!cur[s]) continue;
      /* decode s, add column j's residues, re-encode */
      int64_t rest = s, ns = 0, scale = 1;
      for (int i = 0; i < t; ++i) {
        r[i] = (int32_t)(rest % mods[i]);
        rest /= mods[i];
      }
      for (int i = 0; i < t; ++i) {
        const int32_t ri = (int32_t)((r[i] + A[(size_t)i * n + j] % mods[i]) % mods[i]);
        ns += ri * scale;
        scale *= mods[i];
      }
      nxt[ns] += cur[s]; /* column j taken */
    }
    uint64_t *tmp = cur; cur = nxt; nxt = tmp;
  }
  memcpy(out, cur, sizeof(uint64_t) * (size_t)states);
  free(cur);
  free(nxt);
  return 0;
}
