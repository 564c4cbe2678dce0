/*
 * Drives every oracle function on small seeded instances, for a build with
 * AddressSanitizer and UndefinedBehaviorSanitizer (tests/test_oracle_sanitized.py).
 * The checks here only make the runs meaningful (brute force and meet in the
 * middle agree; histogram totals); the oracle's pins are in test_oracle.py.
 * Exit status 0 and "ok" on stdout when every run agrees.
 */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "../oracle/oracle.h"

static uint64_t rng_state;
static uint64_t next_u64(void) { /* splitmix64: input generation only */
  uint64_t z = (rng_state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

#define MAXN 16
#define MAXM 4
#define CAP (1 << MAXN)

static uint64_t out_b[CAP], out_m[CAP], out_f[CAP];

int main(void) {
  int runs = 0;
  const int ks[3] = {2, 5, 100};
  for (int seed = 1; seed <= 60; ++seed) {
    rng_state = (uint64_t)seed;
    const int m = 1 + (int)(next_u64() % MAXM);
    const int n = 1 + (int)(next_u64() % MAXN);
    const int K = ks[next_u64() % 3];
    int32_t A[MAXM * MAXN], d[MAXM];
    for (int i = 0; i < m * n; ++i) A[i] = (int32_t)(next_u64() % (uint64_t)K);
    const int planted = (int)(next_u64() & 1u);
    uint32_t x = (uint32_t)(next_u64() & ((1u << n) - 1u));
    for (int i = 0; i < m; ++i) {
      int64_t s = 0, row = 0;
      for (int j = 0; j < n; ++j) {
        row += A[i * n + j];
        if (x >> j & 1u) s += A[i * n + j];
      }
      d[i] = (int32_t)(planted ? s : row / 2);
    }
    const int64_t nb = msp_oracle_brute(A, d, m, n, out_b, CAP);
    if (nb < 0 || (planted && nb == 0)) {
      printf("brute failed: seed %d\n", seed);
      return 1;
    }
    for (int slices = 1; slices <= 5; slices += 2) {
      const int64_t nm = msp_oracle_mitm(A, d, m, n, slices, out_m, CAP);
      if (nm != nb || memcmp(out_b, out_m, sizeof(uint64_t) * (size_t)nb) != 0) {
        printf("mitm != brute: seed %d slices %d (%lld vs %lld)\n", seed, slices, (long long)nm, (long long)nb);
        return 1;
      }
      ++runs;
    }
    {
      /* four-list meet in the middle over 0..3 residue rows of small moduli */
      const int t = (int)(next_u64() % (uint64_t)((m < 3 ? m : 3) + 1));
      int32_t fm[3];
      int64_t S = 1;
      for (int k = 0; k < t; ++k) {
        fm[k] = 1 + (int32_t)(next_u64() % 5);
        S *= fm[k];
      }
      uint64_t rec[2];
      const int64_t nf = msp_oracle_fourlist(A, d, m, n, t, fm, 0, S, out_f, CAP, rec, NULL);
      if (nf != nb || memcmp(out_b, out_f, sizeof(uint64_t) * (size_t)nb) != 0 ||
          rec[0] != ((uint64_t)1 << (n / 2)) || rec[1] != ((uint64_t)1 << (n - n / 2))) {
        printf("fourlist != brute: seed %d (%lld vs %lld)\n", seed, (long long)nf, (long long)nb);
        return 1;
      }
      ++runs;
    }
    uint64_t c1[2];
    if (msp_oracle_subset_count(A, n, d[0], c1) != 0) {
      printf("subset_count failed: seed %d\n", seed);
      return 1;
    }
    int32_t cols[MAXN], mods[MAXM];
    for (int j = 0; j < n; ++j) cols[j] = j;
    int64_t states = 1;
    for (int i = 0; i < m; ++i) {
      mods[i] = 1 + (int32_t)(next_u64() % 7);
      states *= mods[i];
    }
    uint64_t hist[7 * 7 * 7 * 7];
    if (msp_oracle_residue_hist(A, m, n, cols, n, m, mods, hist) != 0) {
      printf("residue_hist failed: seed %d\n", seed);
      return 1;
    }
    uint64_t tot = 0;
    for (int64_t s = 0; s < states; ++s) tot += hist[s];
    if (tot != ((uint64_t)1 << n)) {
      printf("residue_hist total %llu != 2^%d: seed %d\n", (unsigned long long)tot, n, seed);
      return 1;
    }
  }
  printf("ok %d runs\n", runs);
  return 0;
}
