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
 *   msp_oracle_fourlist - the same meet in the middle with each half split
 *                        once more (the four lists of Algorithm 1), run
 *                        slice by slice over residue tuples of the first
 *                        rows, so its cost is proportional to the slices it
 *                        enumerates; a slice range gives the solutions whose
 *                        left half lies in those slices.
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
#include <sys/mman.h>
#include <time.h>
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

/* ------------------------------------------------------------------ */
/* Four-list meet in the middle over residue slices (Section 2).       */
/* ------------------------------------------------------------------ */
/*
 * The halves are those of msp_oracle_mitm: left = columns [0, nl) with
 * nl = n/2, right = [nl, n).  Each half of k columns is split once more into
 * an outer part (its first min(FL_OUTER, k/2) columns, more when the inner
 * part would pass FL_INNER columns) and an inner part (the rest): the four
 * lists of Algorithm 1.  A left subset u = (o, i) has the vector
 * v(u) = v(o) + v(i); a right subset w = (o', i') has the target
 * t(w) = d - v(o') - v(i'); (u, w) is a solution exactly when v(u) = t(w)
 * (eq. 1 split between the halves).
 *
 * Slices.  For moduli P_1..P_t of rows 1..t, the slice of a vector y is its
 * residue tuple (y_1 mod P_1, ..., y_t mod P_t), numbered
 * s = r_1 + P_1 (r_2 + P_2 (r_3 + P_3 r_4)).  The slice of a solution x is
 * that of the vector of its left half.  A solution's left vector equals its
 * right target, so both lie in the same slice, and a slice's left subsets
 * need to be joined with that slice's right subsets only.  Residues add: the
 * left subsets of slice r with outer part o are the inner subsets whose
 * residue tuple is r - rho(o) (mod P, row by row), and the right subsets of
 * slice r with outer part o' are the inner subsets with residue tuple
 * d - rho(o') - r.  The inner lists are sorted by residue tuple (bucket) once;
 * a slice reads one bucket per outer subset.
 *
 * Join of one slice: each distinct left vector gets one entry of a hash
 * table (found by a hash of the vector and holding the list of its left
 * subsets); the vectors are recomputed from the subsets whenever a hash
 * matches, so equality is always decided on the full vectors.  Every right
 * target is looked up (one with a negative entry equals no left vector), and
 * every left subset of an equal vector is paired with it.
 *
 * Only slices [s_begin, s_end) are enumerated (all of them give Sol(A, d);
 * any range gives the solutions whose slice lies in it).  records[0] and
 * records[1] receive the left and right subsets the run enumerated (2^nl and
 * 2^(n - nl) over all slices); seconds[0] and seconds[1] (when seconds is
 * not NULL) the wall time of the list build and of the slice joins.
 */
#define FL_INNER 30 /* inner columns per half at most */
#define FL_OUTER 10 /* outer columns per half, when the inner part allows */
#define FL_MAXT 4

typedef struct {
  int t;
  int32_t P[FL_MAXT];
  int64_t stride[FL_MAXT];
  int64_t S;
} fl_slicing;

/* (a + b) mod P and (a - b) mod P for a, b in [0, P) */
static inline int32_t fl_add(int32_t a, int32_t b, int32_t P) { return a + b >= P ? a + b - P : a + b; }
static inline int32_t fl_sub(int32_t a, int32_t b, int32_t P) { return a >= b ? a - b : a - b + P; }

/* A linear 64-bit hash of a vector, H(y) = sum_k c_k y_k mod 2^64 with
 * fixed odd multipliers: H(a + b) = H(a) + H(b) and H(d - a - b) =
 * H(d) - H(a) - H(b), so a subset's hash is the sum of its parts' hashes.
 * Only a filter: equal vectors have equal hashes, and every hash match is
 * decided on the full vectors. */
static inline uint64_t fl_hash(const int32_t *y, int m) {
  uint64_t h = 0, c = 0x9E3779B97F4A7C15ull;
  for (int k = 0; k < m; ++k) {
    h += c * (uint64_t)(int64_t)y[k];
    c = (c * 0xD1342543DE82EF95ull + 0x2545F4914F6CDD1Dull) | 1u;
  }
  return h;
}

/* Table slot of a hash (its top bits after one more multiplication). */
static inline uint64_t fl_slot_of(uint64_t h, int bits) { return (h * 0xBF58476D1CE4E5B9ull) >> (64 - bits); }

/* The subsets of a column range: vectors, residue tuples and hashes, in
 * binary order. */
typedef struct {
  int k;
  int64_t cnt;
  int32_t *vec;   /* [cnt][m] */
  int32_t *res;   /* [cnt][FL_MAXT] */
  uint64_t *hash; /* [cnt] */
} fl_list;

static void fl_list_free(fl_list *l) { free(l->vec); free(l->res); free(l->hash); }

static int fl_list_build(fl_list *l, const int32_t *A, int m, int n, int c0, int k, const fl_slicing *sl) {
  l->k = k;
  l->cnt = (int64_t)1 << k;
  l->vec = (int32_t *)malloc(sizeof(int32_t) * (size_t)(l->cnt * m));
  l->res = (int32_t *)calloc((size_t)(l->cnt * FL_MAXT), sizeof(int32_t));
  l->hash = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)l->cnt);
  if (!l->vec || !l->res || !l->hash) return -2;
  half_t q;
  int32_t v[64];
  half_init(&q, A, m, n, c0, k);
  for (int64_t u = 0; u < l->cnt; ++u) {
    half_step(&q, (uint64_t)u, v);
    memcpy(l->vec + u * m, v, sizeof(int32_t) * m);
    for (int kk = 0; kk < sl->t; ++kk) l->res[u * FL_MAXT + kk] = v[kk] % sl->P[kk];
    l->hash[u] = fl_hash(v, m);
  }
  half_free(&q);
  return 0;
}

/* Large list allocation, backed by huge pages where the kernel offers them
 * on request (fewer TLB misses on the random bucket reads). */
static void *fl_alloc(size_t bytes, int zero) {
  void *p = NULL;
  const size_t align = (size_t)2 << 20;
  bytes = (bytes + align - 1) / align * align;
  if (posix_memalign(&p, align, bytes) != 0) return NULL;
#ifdef MADV_HUGEPAGE
  madvise(p, bytes, MADV_HUGEPAGE);
#endif
  if (zero) memset(p, 0, bytes);
  return p;
}

/* One half's lists.  The outer subsets o; the inner subsets i = (lo, hi),
 * lo its first kl columns and hi the rest, with v(i) = v(lo) + v(hi), sorted
 * by residue tuple: bucket b holds positions [ioff[b], ioff[b + 1]) of imask
 * (the subset bits) and ihash (the hash of v(i)). */
typedef struct {
  int ko, ki, kl;
  fl_list out, lo, hi;
  int64_t ni;
  uint32_t *imask;
  uint64_t *ihash;
  int64_t *ioff; /* [S + 1] */
} fl_half;

static void fl_half_free(fl_half *h) {
  fl_list_free(&h->out); fl_list_free(&h->lo); fl_list_free(&h->hi);
  free(h->imask); free(h->ihash); free(h->ioff);
}

static inline void fl_inner_vec(const fl_half *h, uint32_t i, int m, int32_t *y) {
  const int32_t *a = h->lo.vec + (int64_t)(i & ((1u << h->kl) - 1u)) * m;
  const int32_t *b = h->hi.vec + (int64_t)(i >> h->kl) * m;
  for (int k = 0; k < m; ++k) y[k] = a[k] + b[k];
}

/* Bucket (flattened residue tuple) of inner subset i. */
static inline int64_t fl_inner_bucket(const fl_half *h, const fl_slicing *sl, uint32_t i) {
  const int32_t *a = h->lo.res + (int64_t)(i & ((1u << h->kl) - 1u)) * FL_MAXT;
  const int32_t *b = h->hi.res + (int64_t)(i >> h->kl) * FL_MAXT;
  int64_t s = 0;
  for (int k = 0; k < sl->t; ++k) s += (int64_t)fl_add(a[k], b[k], sl->P[k]) * sl->stride[k];
  return s;
}

/*
 * Counting sort of the inner subsets by bucket, one digit at a time: each
 * thread distributes its share of the subsets into FL_PARTS parts by the
 * bucket's top digit (part p holds buckets [p span, (p + 1) span)), then the
 * parts are sorted by bucket one by one.
 */
#define FL_PARTS 256
static int fl_sort_inner(fl_half *h, const fl_slicing *sl) {
  const int64_t S = sl->S, ni = h->ni;
  const int64_t span = (S + FL_PARTS - 1) / FL_PARTS;
  int nth = 1;
#ifdef _OPENMP
  nth = omp_get_max_threads();
#endif
  int64_t *pc = (int64_t *)calloc((size_t)nth * FL_PARTS, sizeof(int64_t));
  uint32_t *tmp = (uint32_t *)fl_alloc(sizeof(uint32_t) * (size_t)ni, 0);
  if (!pc || !tmp) { free(pc); free(tmp); return -2; }
#pragma omp parallel num_threads(nth)
  {
    int th = 0;
#ifdef _OPENMP
    th = omp_get_thread_num();
#endif
    const int64_t i0 = ni * th / nth, i1 = ni * (th + 1) / nth;
    int64_t *mine = pc + (int64_t)th * FL_PARTS;
    for (int64_t i = i0; i < i1; ++i) ++mine[fl_inner_bucket(h, sl, (uint32_t)i) / span];
#pragma omp barrier
#pragma omp single
    {
      /* cursors: parts in order, threads in order within a part */
      int64_t run = 0;
      for (int p = 0; p < FL_PARTS; ++p)
        for (int q = 0; q < nth; ++q) {
          const int64_t c = pc[(int64_t)q * FL_PARTS + p];
          pc[(int64_t)q * FL_PARTS + p] = run;
          run += c;
        }
    }
    for (int64_t i = i0; i < i1; ++i) tmp[mine[fl_inner_bucket(h, sl, (uint32_t)i) / span]++] = (uint32_t)i;
  }
  /* part p now spans [start(p), start(p + 1)) of tmp; sort each by bucket */
  int64_t pstart[FL_PARTS + 1];
  pstart[0] = 0;
  for (int p = 0; p < FL_PARTS; ++p) pstart[p + 1] = pc[(int64_t)(nth - 1) * FL_PARTS + p];
  int failed = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nth)
  for (int p = 0; p < FL_PARTS; ++p) {
    const int64_t b0 = p * span, b1 = (p + 1) * span < S ? (p + 1) * span : S;
    if (b0 >= b1) continue;
    int64_t *cnt = (int64_t *)calloc((size_t)(b1 - b0 + 1), sizeof(int64_t));
    if (!cnt) {
#pragma omp atomic write
      failed = 1;
      continue;
    }
    const int64_t q0 = pstart[p], q1 = pstart[p + 1];
    for (int64_t q = q0; q < q1; ++q) ++cnt[fl_inner_bucket(h, sl, tmp[q]) - b0 + 1];
    cnt[0] = q0;
    for (int64_t b = b0; b < b1; ++b) cnt[b - b0 + 1] += cnt[b - b0];
    for (int64_t b = b0; b < b1; ++b) h->ioff[b] = cnt[b - b0];
    for (int64_t q = q0; q < q1; ++q) {
      const uint32_t i = tmp[q];
      const int64_t pos = cnt[fl_inner_bucket(h, sl, i) - b0]++;
      h->imask[pos] = i;
      h->ihash[pos] = h->lo.hash[i & ((1u << h->kl) - 1u)] + h->hi.hash[i >> h->kl];
    }
    free(cnt);
  }
  h->ioff[S] = ni;
  free(pc);
  free(tmp);
  return failed ? -2 : 0;
}

static int fl_half_build(fl_half *h, const int32_t *A, int m, int n, int c0, int k, const fl_slicing *sl) {
  memset(h, 0, sizeof(*h));
  h->ko = k / 2 < FL_OUTER ? k / 2 : FL_OUTER;
  if (k - h->ko > FL_INNER) h->ko = k - FL_INNER;
  h->ki = k - h->ko;
  h->kl = h->ki / 2;
  h->ni = (int64_t)1 << h->ki;
  /* outer: columns [c0, c0 + ko); inner low: [c0 + ko, c0 + ko + kl);
   * inner high: [c0 + ko + kl, c0 + k) */
  int rc = fl_list_build(&h->out, A, m, n, c0, h->ko, sl);
  if (rc == 0) rc = fl_list_build(&h->lo, A, m, n, c0 + h->ko, h->kl, sl);
  if (rc == 0) rc = fl_list_build(&h->hi, A, m, n, c0 + h->ko + h->kl, h->ki - h->kl, sl);
  if (rc != 0) return rc;
  h->imask = (uint32_t *)fl_alloc(sizeof(uint32_t) * (size_t)h->ni, 0);
  h->ihash = (uint64_t *)fl_alloc(sizeof(uint64_t) * (size_t)h->ni, 0);
  h->ioff = (int64_t *)fl_alloc(sizeof(int64_t) * ((size_t)sl->S + 1), 0);
  if (!h->imask || !h->ihash || !h->ioff) return -2;
  return fl_sort_inner(h, sl);
}

/* Flattened bucket index of the tuple r - rho (left) or d - rho - r
 * (right, dres = residues of d). */
static inline int64_t fl_bucket(const fl_slicing *sl, const int32_t *r, const int32_t *rho, const int32_t *dres) {
  int64_t b = 0;
  for (int k = 0; k < sl->t; ++k) {
    const int32_t c = dres ? fl_sub(fl_sub(dres[k], rho[k], sl->P[k]), r[k], sl->P[k])
                           : fl_sub(r[k], rho[k], sl->P[k]);
    b += (int64_t)c * sl->stride[k];
  }
  return b;
}

/* Prefetch of an inner bucket's subset bits and hashes (a speed hint only). */
#define FL_AHEAD 4
static inline void fl_prefetch_bucket(const fl_half *h, int64_t b) {
  const int64_t q0 = h->ioff[b], q1 = h->ioff[b + 1];
  for (int64_t q = q0; q < q1; q += 8) __builtin_prefetch(h->ihash + q);
  for (int64_t q = q0; q < q1; q += 16) __builtin_prefetch(h->imask + q);
}

/* A left subset of a slice: its outer subset and inner list position, and
 * the next left subset with the same vector (-1 = none). */
typedef struct {
  uint32_t q;
  int32_t next;
  uint32_t o;
} fl_left;

/* A distinct left vector of a slice: the top 32 bits of its hash and its
 * first left subset (-1 = empty slot). */
typedef struct {
  uint32_t tag;
  int32_t first;
} fl_slot;

/* v(o) + v(i) of a left subset (its outer and inner list entries). */
static inline void fl_left_vec(const fl_half *L, uint32_t o, uint32_t q, int m, int32_t *y) {
  fl_inner_vec(L, L->imask[q], m, y);
  const int32_t *vo = L->out.vec + (int64_t)o * m;
  for (int k = 0; k < m; ++k) y[k] += vo[k];
}

static inline int fl_equal(const int32_t *a, const int32_t *b, int m) {
  for (int k = 0; k < m; ++k)
    if (a[k] != b[k]) return 0;
  return 1;
}

static double fl_now(void) {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

int64_t msp_oracle_fourlist(const int32_t *A, const int32_t *d, int m, int n, int t, const int32_t *mods,
                            int64_t s_begin, int64_t s_end, uint64_t *out, int64_t cap,
                            uint64_t *records, double *seconds) {
  if (records) records[0] = records[1] = 0;
  if (seconds) seconds[0] = seconds[1] = 0.0;
  const double t_start = fl_now();
  if (m < 1 || m > 64 || n < 1 || n > 80 || t < 0 || t > FL_MAXT || t > m) return -1;
  fl_slicing sl;
  sl.t = t;
  sl.S = 1;
  for (int k = 0; k < t; ++k) {
    if (mods[k] < 1) return -1;
    sl.P[k] = mods[k];
    sl.stride[k] = sl.S;
    sl.S *= mods[k];
    if (sl.S > ((int64_t)1 << 28)) return -1;
  }
  if (s_begin < 0 || s_end > sl.S || s_begin > s_end) return -1;
  for (int i = 0; i < m; ++i)
    if (d[i] < 0) return 0;
  for (size_t i = 0; i < (size_t)m * n; ++i)
    if (A[i] < 0) return -1;
  const int words = words_for(n);
  const int nl = n / 2, nr = n - nl;
  int32_t dres[FL_MAXT];
  for (int k = 0; k < t; ++k) dres[k] = d[k] % sl.P[k];
  const uint64_t hd = fl_hash(d, m);
  fl_half H[2];
  int rc = fl_half_build(&H[0], A, m, n, 0, nl, &sl);
  if (rc == 0) rc = fl_half_build(&H[1], A, m, n, nl, nr, &sl);
  if (rc != 0) {
    fl_half_free(&H[0]);
    fl_half_free(&H[1]);
    return rc;
  }
  const fl_half *L = &H[0], *R = &H[1];
  const double t_built = fl_now();
  int64_t count = 0;
  uint64_t recL = 0, recR = 0;
  int failed = 0;

#pragma omp parallel reduction(+ : recL, recR)
  {
    /* per-thread slice buffers, grown as needed */
    int64_t lcap = 0, hcap = 0;
    fl_left *ent = NULL; /* [lcap] left subsets of the slice */
    fl_slot *tab = NULL; /* [hcap] distinct left vectors */
    mask_list found = {0, 0, 0};
    int32_t r[FL_MAXT], y[64], z[64];
    uint64_t mask[MAXW];

    /* consecutive slices read neighbouring buckets: hand them out in runs */
#pragma omp for schedule(dynamic, 64)
    for (int64_t s = s_begin; s < s_end; ++s) {
      int bad;
#pragma omp atomic read
      bad = failed;
      if (bad) continue;
      for (int k = 0; k < t; ++k) r[k] = (int32_t)((s / sl.stride[k]) % sl.P[k]);
      /* left subsets of slice s */
      int64_t cnt = 0;
      for (int64_t o = 0; o < L->out.cnt; ++o) {
        const int64_t b = fl_bucket(&sl, r, L->out.res + o * FL_MAXT, NULL);
        cnt += L->ioff[b + 1] - L->ioff[b];
      }
      for (int64_t o = 0; o < FL_AHEAD && o < R->out.cnt; ++o)
        __builtin_prefetch(R->ioff + fl_bucket(&sl, r, R->out.res + o * FL_MAXT, dres));
      if (cnt >= ((int64_t)1 << 31)) {
#pragma omp atomic write
        failed = 1;
        continue;
      }
      int hbits = 1;
      while (((int64_t)1 << hbits) < 2 * cnt) ++hbits;
      const int64_t hsz = (int64_t)1 << hbits;
      if (cnt > lcap || hsz > hcap) {
        if (cnt > lcap) lcap = cnt;
        if (hsz > hcap) hcap = hsz;
        free(ent); free(tab);
        ent = (fl_left *)malloc(sizeof(fl_left) * (size_t)(lcap + 1));
        tab = (fl_slot *)malloc(sizeof(fl_slot) * (size_t)hcap);
        if (!ent || !tab) {
#pragma omp atomic write
          failed = 1;
          lcap = hcap = 0;
          continue;
        }
      }
      for (int64_t h = 0; h < hsz; ++h) tab[h].first = -1;
      const uint64_t hmask = (uint64_t)hsz - 1;
      int32_t e = 0;
      for (int64_t o = 0; o < L->out.cnt; ++o) {
        const int64_t b = fl_bucket(&sl, r, L->out.res + o * FL_MAXT, NULL);
        const uint64_t ho = L->out.hash[o];
        /* the buckets of later outer subsets: offsets first, then contents */
        if (o + 2 * FL_AHEAD < L->out.cnt)
          __builtin_prefetch(L->ioff + fl_bucket(&sl, r, L->out.res + (o + 2 * FL_AHEAD) * FL_MAXT, NULL));
        if (o + FL_AHEAD < L->out.cnt)
          fl_prefetch_bucket(L, fl_bucket(&sl, r, L->out.res + (o + FL_AHEAD) * FL_MAXT, NULL));
        for (int64_t q = L->ioff[b]; q < L->ioff[b + 1]; ++q, ++e) {
          ent[e].o = (uint32_t)o;
          ent[e].q = (uint32_t)q;
          /* the slot of this left vector: the first empty one, or the one
           * whose tag matches and whose vector is equal */
          const uint64_t hv = ho + L->ihash[q];
          const uint32_t tag = (uint32_t)(hv >> 32);
          int have = 0;
          uint64_t h = fl_slot_of(hv, hbits);
          for (; tab[h].first >= 0; h = (h + 1) & hmask) {
            if (tab[h].tag != tag) continue;
            if (!have) {
              fl_left_vec(L, (uint32_t)o, (uint32_t)q, m, y);
              have = 1;
            }
            const fl_left *f = &ent[tab[h].first];
            fl_left_vec(L, f->o, f->q, m, z);
            if (fl_equal(y, z, m)) break;
          }
          ent[e].next = tab[h].first;
          tab[h].first = e;
          tab[h].tag = tag;
        }
      }
      recL += (uint64_t)cnt;
      /* right subsets of slice s: look up their targets */
      for (int64_t o = 0; o < R->out.cnt; ++o) {
        const int64_t b = fl_bucket(&sl, r, R->out.res + o * FL_MAXT, dres);
        const uint64_t ho = hd - R->out.hash[o];
        if (o + 2 * FL_AHEAD < R->out.cnt)
          __builtin_prefetch(R->ioff + fl_bucket(&sl, r, R->out.res + (o + 2 * FL_AHEAD) * FL_MAXT, dres));
        if (o + FL_AHEAD < R->out.cnt)
          fl_prefetch_bucket(R, fl_bucket(&sl, r, R->out.res + (o + FL_AHEAD) * FL_MAXT, dres));
        recR += (uint64_t)(R->ioff[b + 1] - R->ioff[b]);
        for (int64_t q = R->ioff[b]; q < R->ioff[b + 1]; ++q) {
          const uint64_t hv = ho - R->ihash[q];
          const uint32_t tag = (uint32_t)(hv >> 32);
          int32_t first = -1;
          int have = 0;
          for (uint64_t h = fl_slot_of(hv, hbits); tab[h].first >= 0; h = (h + 1) & hmask) {
            if (tab[h].tag != tag) continue;
            if (!have) { /* the target d - v(o') - v(i') */
              fl_inner_vec(R, R->imask[q], m, y);
              const int32_t *vo = R->out.vec + o * m;
              for (int k = 0; k < m; ++k) y[k] = d[k] - vo[k] - y[k];
              have = 1;
            }
            const fl_left *f = &ent[tab[h].first];
            fl_left_vec(L, f->o, f->q, m, z);
            if (fl_equal(y, z, m)) {
              first = tab[h].first;
              break;
            }
          }
          if (first < 0) continue;
          const uint64_t wsub = (uint64_t)o | ((uint64_t)R->imask[q] << R->ko);
          for (int32_t x = first; x >= 0; x = ent[x].next) {
            const uint64_t usub = (uint64_t)ent[x].o | ((uint64_t)L->imask[ent[x].q] << L->ko);
            memset(mask, 0, sizeof(mask));
            for (int j = 0; j < nl; ++j)
              if ((usub >> j) & 1) set_bit(mask, j);
            for (int j = 0; j < nr; ++j)
              if ((wsub >> j) & 1) set_bit(mask, nl + j);
            if (mask_list_push(&found, mask, words) != 0) {
#pragma omp atomic write
              failed = 1;
              break;
            }
          }
        }
      }
    }
    free(ent); free(tab);
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
  if (seconds) {
    seconds[0] = t_built - t_start;
    seconds[1] = fl_now() - t_built;
  }
  fl_half_free(&H[0]);
  fl_half_free(&H[1]);
  if (records) {
    records[0] = recL;
    records[1] = recR;
  }
  if (failed) return -2;
  if (count <= cap) sort_masks(out, count, words);
  return count;
}
