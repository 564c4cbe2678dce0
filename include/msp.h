/*
 * msp.h - C ABI of libmsp, an exact GPU solver for the feasibility market
 * split problem (n-dimensional subset sum):
 *
 *     find every x in {0,1}^n with  sum_j a_ij x_j = d_i  for i = 1..m
 *
 * (Kempke and Koch, "A GPU accelerated variant of Schroeppel-Shamir's
 * algorithm for solving the market split problem", Section 1, eq. 1.)
 *
 * The columns are split into four quarters whose subset sums are enumerated
 * (Algorithm 1, Section 2).  The key space of the left and right half-pairs
 * is split into residue classes of row 1 or of a surrogate combination of
 * the first rows (eq. 2); only half-pairs of one class can match.  On the
 * direct pass (every instance whose halves have at most 40 columns) a class
 * holds about 2^13 half-pairs per side and one thread block joins it in
 * shared memory; larger instances take the streaming pass, which
 * radix-partitions the half-pairs of a batch of classes through device
 * memory and joins each partition in shared memory.  Every key match is
 * verified exactly on all m rows (Algorithm 2 with the validation of
 * Algorithm 3 and Section 3).
 *
 * Conventions for every entry point:
 *   - All pointers are HOST pointers unless a name says otherwise.  Inputs
 *     are copied during the call; the caller keeps ownership.
 *   - A solution is ceil(n/64) little-endian uint64 words: bit j of word
 *     j/64 is x_j.  Solution lists are sorted ascending as unsigned integers
 *     (most significant word first) and hold no duplicates.  An empty list
 *     (count 0) is a valid result.
 *   - Return values: MSP_OK (0) or MSP_PENDING (1) on success, a negative
 *     msp_status on error; msp_last_error() then describes the error for the
 *     calling thread.  The library never aborts the process and has no CPU
 *     fallback: without a usable CUDA device every solving call fails with
 *     MSP_ECUDA.
 *   - Limits: 1 <= m <= 16, 1 <= n <= 100, a_ij >= 0, d_i >= 0 and every row
 *     sum sum_j a_ij < 65536 (16-bit packed fields).  A right-hand side above
 *     its row sum is accepted and yields no solution.
 *   - libmsp_checked.so (the MSP_CHECKED build) exports the same ABI; its
 *     kernels test their data-dependent indices before each access, skip an
 *     access that fails, and the solve then returns MSP_ECUDA naming the
 *     check (msp_version() names the build).
 */
#ifndef MSP_H
#define MSP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MSP_API __attribute__((visibility("default")))
#else
#define MSP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MSP_OK = 0,
  MSP_PENDING = 1,     /* msp_poll: request not finished yet */
  MSP_EINVAL = -1,     /* bad argument (null pointer, negative entry, bad handle) */
  MSP_ERANGE = -2,     /* outside the limits above */
  MSP_ENOMEM = -3,     /* device or host allocation failed / budget too small */
  MSP_ECUDA = -4,      /* a CUDA call failed (no device, launch error, ...) */
  MSP_ETIMEDOUT = -5,  /* a bounded device wait gave up */
  MSP_EOVERFLOW = -6,  /* result or intermediate list larger than supported */
  MSP_ECANCELED = -7   /* request canceled before completion */
} msp_status;

typedef struct msp_instance msp_instance; /* one (A, d); owns its device state */
typedef struct msp_server msp_server;     /* request queue + device scheduler   */

/* Per-solve counters, filled by msp_solve_all and readable afterwards. */
typedef struct {
  int m, n;
  int quarter[4];             /* quarter sizes q1..q4 (L = Q1+Q3, R = Q2+Q4) */
  int class_bits;             /* residue classes: 2^class_bits               */
  int class_rows;             /* rows combined in the residue key (1 = row 1) */
  int digit_bits;             /* radix-partition digit of the pass sort       */
  int passes;                 /* residue passes run                           */
  uint64_t records_left;      /* |L| = 2^(q1+q3) half-pair records            */
  uint64_t records_right;     /* |R| = 2^(q2+q4)                              */
  uint64_t row1_candidates_lo;/* C1: pairs (l, r) with row1(l)+row1(r) = d1,  */
  uint64_t row1_candidates_hi;/*     as a 128-bit integer (hi:lo)             */
  uint64_t key_matches;       /* distinct matched keys checked exactly        */
  uint64_t pairs_verified;    /* candidate quadruples checked on all m rows   */
  uint64_t solutions;         /* distinct solutions                          */
  uint64_t oversize_segments; /* partitions joined by the general path        */
  uint64_t device_bytes;      /* peak device memory of the solve              */
  double ms_total;            /* wall time of the last msp_solve_all          */
  uint64_t kernel_launches;   /* kernels launched by the last solve           */
  uint64_t fast_passes_redone;/* streaming passes re-run on the exact path    */
  uint64_t h2d_bytes;         /* host-to-device bytes copied by the solve     */
  uint64_t d2h_bytes;         /* device-to-host bytes copied by the solve     */
  uint64_t classes_total;     /* residue classes of the instance (2^class_bits) */
  uint64_t classes_done;      /* classes this solve enumerated                */
  uint64_t records_done;      /* half-pair records (both sides) it generated   */
  int path;                   /* pass that solved it: 0 streaming / exact, 1 direct */
  int direct_fallback;        /* 1: the direct pass handed the solve to the others */
  /* Filled only when profiling is on (msp_set_profiling): per kernel kind
   * (MSP_K_* below) the summed CUDA-event time, the launches, and the
   * algorithmic device-memory bytes (records written / read x 8 bytes). */
  double kernel_ms[12];
  uint64_t kernel_count[12];
  uint64_t kernel_bytes[12];
} msp_stats;

/* Kernel kinds indexing msp_stats.kernel_* */
enum {
  MSP_K_GRAY = 0,      /* quarter lists by Gray code                 */
  MSP_K_BUCKET = 1,    /* residue-class counting sort                */
  MSP_K_C1 = 2,        /* row-1 candidate count                      */
  MSP_K_GEN_COUNT = 3, /* partition histograms of a pass             */
  MSP_K_OFFSETS = 4,   /* histograms to offsets                      */
  MSP_K_GEN_SCATTER = 5, /* records generated and radix-partitioned  */
  MSP_K_JOIN = 6,      /* shared-memory sort + merge-join            */
  MSP_K_JOIN_BIG = 7,  /* oversize partitions                        */
  MSP_K_RECOVER = 8,   /* quarter elements behind matched keys       */
  MSP_K_VERIFY = 9,    /* exact all-row check                        */
  MSP_K_OTHER = 10,
  MSP_K_DIRECT = 11    /* direct pass: class joins in shared memory   */
};

/* Validate and copy (A row-major m x n, d length m); upload to the device.
 * A and d are the matrix and right-hand side of the system A x = d over
 * x in {0,1}^n (Section 1, eq. 1; a_ij and d_i in N0).  On success *out owns
 * the instance (free with msp_destroy). */
MSP_API int msp_create(const int32_t *A, const int32_t *d, int m, int n, msp_instance **out);

/* Release an instance and its device memory (NULL is ignored). */
MSP_API void msp_destroy(msp_instance *inst);

/* Run work of this instance on the given CUDA stream (a cudaStream_t passed
 * as void*; NULL = the library's own stream for this instance). */
MSP_API int msp_set_stream(msp_instance *inst, void *cuda_stream);

/* Cap the device memory one solve may use (bytes; 0 = 85% of free memory). */
MSP_API int msp_set_memory_budget(msp_instance *inst, size_t bytes);

/* Instance options (msp_set_option):
 *   MSP_OPT_EXACT_PATH  1 = skip the direct and streaming passes and run
 *                       every residue pass on the exact two-phase path
 *                       (count, then scatter); 0 = default (direct pass when
 *                       the instance fits it, else streaming with an exact
 *                       re-run of any pass whose partitions overflow). */
/*   MSP_OPT_CLASS_PART, MSP_OPT_CLASS_PARTS  enumerate only the residue
 *                       classes [k*M/P, (k+1)*M/P) of the M classes, with
 *                       k = PART and P = PARTS (default 0 of 1: all).  The
 *                       solutions of the P parts are disjoint and their union
 *                       is the full solution set, so parts can be solved by
 *                       different processes or GPUs, or one part timed to
 *                       project the full time (records_done / all records). */
/*   MSP_OPT_CLASS_BITS   residue classes 2^B of the plan, B in [0, 27]
 *   MSP_OPT_DIGIT_BITS   radix digit bits D of the streaming pass, in [0, 12]
 *                        (partitions of about |L| / 2^(B + D) records; a class
 *                        whose partitions would not fit shared memory is
 *                        solved on the exact path)
 *   MSP_OPT_INNER_BITS   the inner quarter of each side (Q3 of L, Q4 of R)
 *                        gets B + value columns (at most 27, or 30 when B is
 *                        above 23 or a half has 44 columns or more; never
 *                        fewer than the even split; the formula takes 4, or 5
 *                        for halves of 44 to 47 columns), so an
 *                        inner residue bucket holds
 *                        about 2^value elements: the run of records one outer
 *                        element expands to in the scatter, in [0, 12]
 *                        For these three, -1 (the default) restores the
 *                        built-in formula; any choice gives the same solutions.
 *                        They are what the package's autotuner sets per (m, n). */
/*   MSP_OPT_DIRECT       the direct pass (default for every instance it
 *                        fits: halves of at most 40 columns): the columns of
 *                        each half are split into an outer quarter of at most
 *                        2^9 subsets and an inner quarter bucketed into
 *                        residue classes of about 16 subsets, so a thread
 *                        block joins a whole class (about 2^13 records per
 *                        side) in shared memory and no record is written to
 *                        device memory.  1 = use it whenever the instance fits
 *                        (the three streaming-pass options above are then
 *                        ignored), 0 = never, -1 (default) = use it unless one
 *                        of the three streaming-pass options is set.
 *   MSP_OPT_TABLE_BITS   shared hash table of the direct pass: 2^value slots,
 *                        value in [12, 15]; -1 = 14.
 *                        Either choice gives the same solutions.
 *   MSP_OPT_FIRST        1 = time to first solution (the quantity the paper's
 *                        Algorithm 2 returns): on the direct pass the residue
 *                        classes are joined in launches of about 2^32
 *                        records, the matches verified after each, and the
 *                        solve stops after the first launch that yields a
 *                        solution.  The streaming pass likewise verifies the
 *                        matches after every residue pass and stops after
 *                        the first pass that yields a solution (the exact
 *                        re-runs of overflowed passes come only after all
 *                        streaming passes).  The result is then a nonempty
 *                        subset of the solutions (all of those found so far)
 *                        and msp_stats.classes_done counts the classes
 *                        joined; an instance with no solution is still
 *                        searched to the end.  0 = every solution
 *                        (default). */
enum {
  MSP_OPT_EXACT_PATH = 1,
  MSP_OPT_CLASS_PART = 2,
  MSP_OPT_CLASS_PARTS = 3,
  MSP_OPT_CLASS_BITS = 4,
  MSP_OPT_DIGIT_BITS = 5,
  MSP_OPT_INNER_BITS = 6,
  MSP_OPT_DIRECT = 7,
  MSP_OPT_TABLE_BITS = 8,
  MSP_OPT_FIRST = 9,
  MSP_OPT_WAIT_LIMIT_US = 10,
  MSP_OPT_WAIT_CHECK = 11
};
/*   MSP_OPT_WAIT_LIMIT_US  limit of each bounded wait of the streaming pass's
 *                        join for a bulk copy, in microseconds, in [1, 6e7]
 *                        (default 2e6, i.e. 2 s).  A wait that runs out sets
 *                        an error flag, waits once more (bounded by the same
 *                        limit) so that the copy lands before its block
 *                        exits, and the solve returns MSP_ETIMEDOUT.
 *   MSP_OPT_WAIT_CHECK   1 = check of that path: before its first copy, every
 *                        block of the streaming join waits on a barrier phase
 *                        that no copy completes, so the wait runs out and the
 *                        solve returns MSP_ETIMEDOUT (with nothing in flight);
 *                        the device and the library stay usable.  0 = off
 *                        (default).  Neither changes any result. */
MSP_API int msp_set_option(msp_instance *inst, int option, int64_t value);

/* Time every kernel launch of later solves with CUDA events (on = 1). */
MSP_API int msp_set_profiling(msp_instance *inst, int on);

/* Exhaustive solve: every x with A x = d, the set of Section 1, eq. 1 (the
 * paper's Algorithm 2 stops at the first; this call returns all of them
 * unless MSP_OPT_FIRST is set).  The four quarter lists of Algorithm 1 are
 * built on the device, the half-pairs joined by residue class (eq. 2's
 * surrogate idea as the class key) and every key match checked on all m rows
 * (Algorithm 3's validation).  Blocking.  *masks is allocated by the library
 * (free with msp_free_solutions; NULL when *count is 0); *words_per_mask is
 * ceil(n/64).  Errors: MSP_EINVAL (null argument), MSP_ENOMEM (the memory
 * budget holds no pass), MSP_ECUDA, MSP_ETIMEDOUT, MSP_EOVERFLOW,
 * MSP_ECANCELED (serving loop only). */
MSP_API int msp_solve_all(msp_instance *inst, uint64_t **masks, size_t *count, int *words_per_mask);

/* Counters of the last solve of this instance. */
MSP_API int msp_get_stats(const msp_instance *inst, msp_stats *out);

/* Free a solution buffer returned by this library (NULL is ignored). */
MSP_API void msp_free_solutions(uint64_t *masks);

/* Solve `count` independent instances of the same (m, n): A[k] and d[k]
 * point to instance k, and its result is eq. 1's set for (A[k], d[k]) (the
 * paper solves one instance at a time; batching has no counterpart there).  Solutions of instance k are masks[offsets[k] ..
 * offsets[k+1]) in units of masks (each ceil(n/64) words); offsets has
 * count+1 entries; *masks is library-allocated (msp_free_solutions). */
MSP_API int msp_solve_batch(const int32_t *const *A, const int32_t *const *d, int m, int n, int count,
                    uint64_t **masks, size_t *offsets);

/* msp_solve_batch with the enumeration path chosen: path 1 = the direct pass
 * (MSP_ERANGE when the instances do not fit it), 0 = the streaming pass,
 * -1 = the direct pass when it fits, else streaming (what msp_solve_batch
 * does).  On the direct pass every instance's lists are built, then the
 * residue classes of all instances are joined by one launch (per 2^20
 * classes) and every match is verified by one more. */
MSP_API int msp_solve_batch_path(const int32_t *const *A, const int32_t *const *d, int m, int n, int count,
                                 int path, uint64_t **masks, size_t *offsets);

/* Serving: a request queue whose instances share the device (no counterpart
 * in the paper; each request's result is eq. 1's set for its instance, the
 * same as msp_solve_all's).  Requests are admitted while their device
 * footprint fits the memory budget, and the passes of admitted requests are
 * interleaved on several streams.
 *   msp_server_create: hbm_budget_bytes 0 = 80% of the free device memory;
 *     max_inflight in [1, 64] workers.  MSP_ECUDA without a device.
 *   msp_submit: A, d as for msp_create, copied; *req_id identifies the
 *     request.  MSP_ENOMEM when its footprint exceeds the whole budget.
 *   msp_cancel: a queued request is dropped, a running one stops at its next
 *     launch boundary; its msp_poll then returns MSP_ECANCELED. */
MSP_API int msp_server_create(size_t hbm_budget_bytes, int max_inflight, msp_server **out);
MSP_API int msp_submit(msp_server *srv, const int32_t *A, const int32_t *d, int m, int n, uint64_t *req_id);
/* MSP_PENDING while running; MSP_OK with the solutions once done (masks as in
 * msp_solve_all, then the request is forgotten); a negative status on error. */
MSP_API int msp_poll(msp_server *srv, uint64_t req_id, uint64_t **masks, size_t *count, int *words);
MSP_API int msp_cancel(msp_server *srv, uint64_t req_id);
MSP_API void msp_server_destroy(msp_server *srv);

/* Exhaustive solve of a small instance (n <= 40) that allocates no device
 * memory.  The paper has no counterpart: it is for callers that cannot
 * allocate device memory while solving - a process whose device memory is
 * owned (and possibly fully reserved) by another framework's allocator, a
 * serving loop that must not risk an out-of-memory failure or an allocator
 * stall mid-request, or code running under a fixed device-memory quota.
 * It runs the same kernels as msp_solve_all (the exact two-phase residue
 * pass) with every intermediate buffer taken from one static device array of
 * 24 MiB that each device holding the library keeps until process exit.
 *   A (m x n row-major) and d (m): host inputs, copied during the call.
 *   masks: caller-owned host buffer of `cap` uint64 (one word per solution,
 *   since n <= 40); on MSP_OK it holds *count sorted distinct solutions.
 *   stream: cudaStream_t (as void*) to run on; NULL = the legacy stream.
 *   Errors: MSP_ERANGE for n > 40 (and the usual limits), MSP_EOVERFLOW when
 *   the solutions exceed `cap` (then *count is an upper bound to retry with)
 *   or the static scratch (more than 8192 matched keys, 131072 candidates or
 *   131072 solutions).
 * Every call looks up the array's address on the caller's current device, so
 * a device reset between calls is harmless.  The call synchronises `stream`
 * (it reads counts back between its phases), so it must not be made while
 * that stream is capturing a CUDA graph.  All calls share the array, so calls
 * that overlap on the GPU race: serialise them. */
MSP_API int msp_solve_small_noalloc(const int32_t *A, const int32_t *d, int m, int n, uint64_t *masks,
                                    size_t cap, size_t *count, void *stream);

/* Thread-local description of the last error (never NULL). */
MSP_API const char *msp_last_error(void);

/* Library version string. */
MSP_API const char *msp_version(void);

/* Name of the calling thread's current CUDA device ("" when there is none);
 * the autotuner keys its cache by it. */
MSP_API const char *msp_device_name(void);

/* The plan msp_solve_all takes by default for an (m, n) instance, computed
 * on the host (no device is needed; the memory check of a solve may still
 * hand a direct-pass instance to the streaming pass). */
typedef struct {
  int path;              /* 1 = direct pass, 0 = streaming pass                  */
  int class_bits;        /* residue classes: 2^class_bits                         */
  int class_rows;        /* rows combined in the residue key                      */
  int quarter[4];        /* q1..q4, L = Q1+Q3, R = Q2+Q4 (direct pass: outer L,
                            outer R, inner L, inner R), as in msp_stats           */
  int digit_bits;        /* streaming pass: radix digit bits (direct pass: 0)     */
  int table_bits;        /* direct pass: 2^table_bits table slots (streaming: 0)  */
  uint64_t records_left;  /* |L| = 2^(q1+q3)                                      */
  uint64_t records_right; /* |R| = 2^(q2+q4)                                      */
  uint64_t device_bytes;  /* estimated device memory of a solve, uncapped         */
} msp_plan_info;
/* MSP_OK, MSP_EINVAL (out is null) or MSP_ERANGE (m outside [1, 16] or n
 * outside [1, 100]). */
MSP_API int msp_plan(int m, int n, msp_plan_info *out);

#ifdef __cplusplus
}
#endif

#endif /* MSP_H */
