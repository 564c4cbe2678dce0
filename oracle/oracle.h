/*
 * CPU oracle for the feasibility market split problem.  TEST INFRASTRUCTURE
 * ONLY: used by the tests, the package smoke check and the benchmark's CPU
 * baseline, never by the product path.  See oracle.c for what each function
 * computes and which passage of the paper it follows.
 */
#ifndef MSP_ORACLE_H
#define MSP_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif
int msp_oracle_words(int n);
int64_t msp_oracle_brute(const int32_t *A, const int32_t *d, int m, int n, uint64_t *out, int64_t cap);
int64_t msp_oracle_mitm(const int32_t *A, const int32_t *d, int m, int n, int slices, uint64_t *out,
                        int64_t cap);
int64_t msp_oracle_fourlist(const int32_t *A, const int32_t *d, int m, int n, int t, const int32_t *mods,
                            int64_t s_begin, int64_t s_end, uint64_t *out, int64_t cap, uint64_t *records,
                            double *seconds);
int msp_oracle_subset_count(const int32_t *w, int n, int64_t target, uint64_t out[2]);
int msp_oracle_residue_hist(const int32_t *A, int m, int n, const int32_t *cols, int ncols, int t,
                            const int32_t *mods, uint64_t *out);
#ifdef __cplusplus
}
#endif
#endif
