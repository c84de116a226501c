/*
 * dist.h -- C ABI of libdist: exact symplectic minimum distance on one GB300.
 *
 * Problem (Section 2, definitions of wt_s and wt_s(C)): for an F2-linear code
 * C in F2^{2n} given by generator rows (x | z),
 *     d = min { wt_s(c) : c in C, c != 0 },   wt_s(x, z) = popcount(x OR z).
 * An F4-linear code of length n (Section 2.3) is the same problem: its F4
 * Hamming weight equals wt_s of the 2-bit-plane image a + alpha b -> (a | b).
 *
 * Method (Section 2.1, Brouwer-Zimmermann with the packages of Sections 2.2
 * and 2.3): the code is put into systematic generator matrices Gamma_1..m on
 * disjoint qubit sets; for r = 1, 2, ... every combination of r units
 * (packages of rows sharing a pivot qubit, or free rows) of every included
 * matrix is enumerated on the GPU; the smallest weight seen is the upper
 * bound U, and the lower bound L = sum_j max(0, r + 1 - f_j) (f_j = free rows
 * of Gamma_j; Section 2.3's bound for two matrices, generalised) rises after
 * every round; d = U once L >= U.
 *
 * Steps of the path (the labels S1-S7 used in the sources):
 *   S1 ingest: validate the rows, pack the bit-planes, reduce to full rank;
 *   S2 diagonalize: the matrices Gamma_j and their units;
 *   S3 bounds: L after every (round, matrix) step, the matrices included;
 *   S4 enumerate: every combination of a round, on the GPU;
 *   S5 reduce: the running minimum U and the witness slot of each weight;
 *   S6 certify: stop once L >= U, rebuild and check the witness;
 *   S7 batch and serve: many codes per launch, continuous admission.
 *
 * Conventions:
 *   - Every function returns DIST_OK (0) or a negative DIST_E* code; nothing
 *     throws across the ABI.  dist_strerror() names a code.
 *   - Inputs are plain host pointers and are copied; the caller keeps them.
 *   - Outputs go into caller-allocated structs.
 *   - A dist_code is used by one host thread at a time.
 *   - The library needs a CUDA device (sm_103a build).  Without one, calls
 *     that touch the device return DIST_ECUDA; there is no CPU fallback.
 *   - cuda_stream arguments are cudaStream_t values passed as void*; NULL
 *     selects a stream owned by the dist_code.
 */
#ifndef DIST_H
#define DIST_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { DIST_F2 = 2, DIST_F4 = 4 };

enum {
    DIST_OK = 0,
    DIST_EINVAL = -1,      /* bad argument or input outside the limits below */
    DIST_ENOMEM = -2,      /* host or device allocation failed */
    DIST_ECUDA = -3,       /* CUDA error, or no usable device */
    DIST_ETIMEOUT = -4,    /* a bounded wait ran out */
    DIST_EINCOMPLETE = -5, /* time limit reached: lower <= d <= upper in the result */
    DIST_EZERO = -6,       /* the code (or C minus S) has no nonzero codeword */
    DIST_EBUSY = -7,       /* batch ticket not finished yet */
    DIST_EINTERNAL = -8,   /* a self-check of the library failed */
    DIST_ERANGE = -9       /* distance needs combinations beyond the device walk (r > 32) */
};

#define DIST_MAX_N 128     /* qubits */
#define DIST_MAX_K 256     /* F2 rows (an F4 input counts twice) */

typedef struct dist_code dist_code;

/*
 * dist_init -- ingest and diagonalize a code (steps S1-S2; Section 2.2,
 * Diagonalization_over_F2, and Section 2.3, Diagonalization_over_F4), and
 * upload its generator matrices to the current CUDA device.
 *   generator: field DIST_F2 -> K rows x 2n bytes in {0,1}, row-major, each
 *              row x_0..x_{n-1} | z_0..z_{n-1}.
 *              field DIST_F4 -> K rows x n bytes in {0,1,2,3}; v = a + 2b
 *              means a + alpha b with alpha^2 = alpha + 1 (x-plane a,
 *              z-plane b).  The code is the F4-span of the rows.
 *   1 <= n <= 128; 1 <= K; K <= 256 (F2) or 2K <= 256 (F4).
 *   Rank-deficient input is reduced (k_eff in the result); rank 0 gives
 *   DIST_EZERO.  On success *out owns host and device memory until
 *   dist_free.
 */
int dist_init(dist_code **out, const uint8_t *generator, int n, int K, int field);

/*
 * dist_init_many -- dist_init of count codes in one call (steps S1-S2 for a
 * batch, Sections 2.2-2.3): the codes are ingested and diagonalized on the
 * library's host threads (one per hardware thread beyond the caller's, at
 * most 15), and their device blocks are carved from one allocation, which
 * is freed with the last of its codes.
 *   out[i]:                      the code (NULL where status[i] < 0).
 *   generators[i], n[i], K[i], field[i]: as dist_init (host memory, read
 *                                during the call).
 *   status[i]:                   DIST_OK or the error dist_init would return.
 * Every array has count entries; count = 0 is accepted.  Returns DIST_OK if
 * every code was initialised, else the status of the first that was not
 * (the others are initialised and must be released with dist_free).
 * DIST_EINVAL if count < 0 or an array is NULL.
 */
int dist_init_many(dist_code **out, int count, const uint8_t *const *generators, const int *n, const int *K,
                   const int *field, int *status);

/*
 * dist_set_exclude -- take the minimum over C minus S, S = span of the first
 * n_stab input rows (F4: their F4-span).  With a normalizer matrix whose
 * first rows generate the stabilizer this is d(Q) = wt_s(N \ S), the check of
 * the modified Brouwer-Zimmermann algorithm (Section 2.1).  n_stab = 0
 * restores the plain minimum.  DIST_EZERO if S = C.
 */
int dist_set_exclude(dist_code *c, int n_stab);

typedef struct {
    int32_t d;            /* certified distance (upper bound U if incomplete) */
    int32_t lower;        /* lower bound on d (= d when certified) */
    int32_t rounds;       /* last combination size r enumerated */
    int32_t k_eff;        /* rank of the input (F4: over F4) */
    int32_t n_gamma;      /* generator matrices enumerated */
    int32_t status;       /* DIST_OK, DIST_EINCOMPLETE, ... (same as return) */
    uint64_t codewords;   /* (subset, representative) combinations evaluated */
    double seconds;       /* host wall time of the call */
    uint8_t witness[256]; /* a codeword of weight d: F2 2n bytes (x | z), F4 n symbols */
    uint8_t coeffs[256];  /* its coefficients over the input rows: F2 bits, F4 symbols */
    double gpu_seconds;   /* summed run time of the enumeration kernels (dist_set_event_timing) */
    uint64_t launches;    /* enumeration kernels launched */
} dist_result;

/*
 * dist_solve -- steps S3-S6, the Brouwer-Zimmermann loop of Section 2.1 with
 * the package bound of Section 2.3: for r = 1, 2, ... every r-subset of the
 * units of each enumerated generator matrix, every representative choice
 * (F4: the first unit's scalar fixed to 1), weighed by wt_s = popcount(x OR
 * z); the upper bound U is the lightest codeword met (outside S with
 * dist_set_exclude), the lower bound L = sum_j max(0, r + 1 - f_j) over the
 * finished rounds (f_j: free rows of matrix j), and d = U once L >= U.
 *   c:           from dist_init; used by one host thread at a time.
 *   out:         caller-owned; filled completely (d, witness, coefficients,
 *                counts, times).  witness is re-checked on the host against
 *                the input rows before DIST_OK is returned.
 *   cuda_stream: a cudaStream_t (NULL: the library's own stream); work is
 *                ordered on it and the call returns after the result is on
 *                the host.
 * Errors: DIST_EINVAL (NULL arguments), DIST_EBUSY (c is in a batch),
 * DIST_EZERO (no nonzero codeword outside S), DIST_ERANGE (certification
 * needs combinations beyond the device walk), DIST_ECUDA, DIST_EINTERNAL (a
 * witness failed the host re-check; no d is returned).
 */
int dist_solve(dist_code *c, dist_result *out, void *cuda_stream);

/*
 * dist_solve_bounded -- as dist_solve (Section 2.1), but stops after about
 * time_limit_s seconds and then returns DIST_EINCOMPLETE with certified
 * bounds lower <= d <= upper (out->d = upper, out->witness of weight upper).
 * The limit is checked between launches and by the kernel itself (a
 * %globaltimer budget); a launch that ends on its budget certifies d only if
 * U already met the bound that held before it.  time_limit_s <= 0 means no
 * limit (dist_solve).
 */
int dist_solve_bounded(dist_code *c, dist_result *out, void *cuda_stream, double time_limit_s);

/* dist_free -- releases a dist_code (NULL is accepted). */
int dist_free(dist_code *c);

/*
 * dist_solve_isometry -- the same distance by the paper's isometry method
 * (Algorithm 3, Saved_isometry) on the GPU, for comparison with the package
 * method: the image (a, b, a + b) in F2^{3n} is searched with plain binary
 * Brouwer-Zimmermann over systematic matrices on disjoint information sets
 * (later ones may have deficient rank), one launch per (round, matrix).  The
 * Hamming weight of the image is twice the symplectic weight, so d = U / 2.
 * Exclusion (dist_set_exclude) applies.  Results as dist_solve; codewords
 * counts binary combinations (rows of the image), n_gamma its matrices.
 * DIST_ERANGE if certification needs more than 32 rows per combination.
 */
int dist_solve_isometry(dist_code *c, dist_result *out, void *cuda_stream);
/*
 * Which walk dist_solve_isometry runs on rounds r >= 2 (process-wide).
 * 0 (the default): the split walk (rows cut into two halves, every r-subset a
 * product of one subset of each) on rounds of at most 8 rows with at least
 * 2^18 combinations, the pair-table walk on the other rounds whose table fits
 * in shared memory, the revolving-door lane walk elsewhere.  1: the split
 * walk on every round r in [2, 8].  2: never the split walk.  Affects speed,
 * never results.  DIST_EINVAL for other values.
 */
int dist_set_iso_walk(int mode);
int dist_get_iso_walk(void);

/*
 * Batched and served solving (step S7; the paper has no counterpart -- its
 * parallel version splits one code's combinations over CPU threads).
 *
 * A dist_batch runs many dist_codes on one device together: one launch of
 * the multi-code enumeration kernel serves every admitted code, each code
 * keeping its bound, chunk counter and witness slots on the device between
 * launches.  A worker thread owned by the batch runs time-bounded "slices",
 * each one replay of a captured CUDA graph (one upload of the slice's arena,
 * scratch set-up, the multi-code launch, gather, one read-back); codes
 * submitted while others run are admitted at the next slice boundary
 * (continuous batching), subject to max_active and max_resident_bytes (the
 * codes' device footprint: tables + scratch).  A dist_batch is internally
 * synchronized: any thread may submit, poll or wait.  A submitted dist_code
 * belongs to the batch until its ticket has been collected by poll or wait:
 * dist_solve / dist_free on it return DIST_EBUSY meanwhile.
 */
typedef struct {
    int32_t max_active;          /* codes on the device at once (0 = 8192) */
    int32_t pad;
    double slice_ms;             /* time budget of one launch in ms; 0 = none (run to completion) */
    uint64_t max_resident_bytes; /* admission limit on the active codes' footprint (0 = none) */
    double time_limit_s;         /* per code, from admission; 0 = none.  A code that reaches it
                                    ends with status DIST_EINCOMPLETE and lower <= d <= d(upper) */
} dist_batch_opts;

typedef struct {
    uint64_t slices, launches, codes_done, active, pending, resident_bytes;
    double gpu_seconds;          /* summed CUDA-event time of the multi-code launches */
    double plan_seconds;         /* worker time before the launches: planning and packing */
    double post_seconds;         /* worker time after them: read-back wait, verdicts, witnesses */
} dist_batch_stats_t;

typedef struct dist_batch dist_batch;

/* Creates a batch on the current device; opts may be NULL (defaults).  It
 * allocates the batch's 32 MB staging arena (pinned host and device memory;
 * larger slices grow it) and captures its slice graph, so that the first
 * slices allocate nothing. */
int dist_batch_create(dist_batch **b, const dist_batch_opts *opts);
/* Queues count codes (initialised with dist_init on the same device) as one ticket. */
int dist_batch_submit(dist_batch *b, dist_code *const *codes, int count, uint64_t *ticket);
/* DIST_EBUSY until every code of the ticket is done; then fills results[count]
 * (per-code status in results[i].status; seconds = latency from submission)
 * and releases the ticket. */
int dist_batch_poll(dist_batch *b, uint64_t ticket, dist_result *results);
/* As poll, blocking up to timeout_s seconds (<= 0: no limit); DIST_ETIMEOUT on expiry. */
int dist_batch_wait(dist_batch *b, uint64_t ticket, dist_result *results, double timeout_s);
/* Waits up to timeout_s (<= 0: no limit) for any submitted ticket to finish and
 * returns its id in *ticket (collect it with poll); each finished ticket is
 * reported once.  DIST_ETIMEOUT on expiry. */
int dist_batch_wait_any(dist_batch *b, double timeout_s, uint64_t *ticket);
int dist_batch_stats(dist_batch *b, dist_batch_stats_t *stats);
/* Stops the worker after its current slice and frees the batch; uncollected
 * tickets are dropped and their codes released. */
int dist_batch_destroy(dist_batch *b);

/*
 * Chunk granularity of the enumeration launches (process-wide; affects
 * speed, never results).  chunks_per_warp: each enumeration step is cut
 * into about this many warp-chunks per resident warp (default 6, range
 * 1..256); a lane chunk holds at most 2^lane_cap_log2 (default 14, range
 * 8..24) codewords, and a fast-path segment at least 2^lane_floor_log2
 * (default 12, range 1..lane_cap_log2) unless that would leave it fewer
 * chunks than resident warps; outside a launch's last step a fast-path lane
 * chunk also holds at least eight subsets.  Values outside the ranges are
 * clamped; fields <= 0 keep the current value.  dist_autotune times calibration solves (random codes of
 * 64 x 56 and 72 x 72) on the current device over a grid of the three,
 * applies the setting with the best geometric-mean codewords/s (the setting
 * in force stays unless another is at least 2 % faster; a setting that cuts
 * every launch of the codes exactly as one already timed is not timed
 * again), and returns it (and that rate) -- about budget_s seconds (<= 0:
 * about 10 s).
 */
typedef struct {
    int32_t chunks_per_warp;
    int32_t lane_cap_log2;
    int32_t lane_floor_log2;
    double codewords_per_s;      /* dist_autotune: rate of the chosen setting */
} dist_tuning;
int dist_set_tuning(const dist_tuning *t);
int dist_get_tuning(dist_tuning *t);
int dist_autotune(dist_tuning *best, double budget_s);
/* The tuning search of dist_autotune, timed on the caller's codes
 * (initialised on the current device, not in a batch): tunes for a known
 * workload. */
int dist_autotune_codes(dist_code *const *codes, int count, double budget_s, dist_tuning *best);
/*
 * Information-set search of the planner (process-wide): for a code whose
 * estimated work exceeds 5e8 codewords and whose enumerated matrices have
 * free rows, dist_init also diagonalizes with up to `trials` seeded random
 * qubit orders and keeps the plan with the least estimated work (0 = index
 * order only; default 8; range 0..256).  Affects speed, never results.
 */
int dist_set_plan_search(int trials);
int dist_get_plan_search(void);
/*
 * Matrix-inclusion limit of the planner (process-wide; Section 2.3, the
 * second generator matrix and its bound term): dist_init enumerates at most
 * `m` of the generator matrices it builds on disjoint qubit sets, the prefix
 * (by free rows) with the least estimated work (0 = no limit, the default;
 * 1 = the first matrix only, as a one-matrix Brouwer-Zimmermann does).
 * Affects speed, never results.  DIST_EINVAL for m < 0; values above 16 act
 * as 16.
 */
int dist_set_gamma_limit(int m);
int dist_get_gamma_limit(void);
/*
 * How gpu_seconds of dist_solve, dist_solve_bounded and dist_solve_noalloc
 * is measured (process-wide).  0 (the default): by the enumeration kernel
 * itself, from the earliest block start to the latest warp end of each
 * launch (%globaltimer, 32 ns steps), at no cost.  1: by CUDA events
 * recorded on the solve's stream around each launch (not for
 * dist_solve_noalloc, which creates no events); a timed event pair adds
 * about 11 us to each launch on a GB300.  Never affects results.
 */
int dist_set_event_timing(int on);
int dist_get_event_timing(void);

/*
 * dist_plan_info -- host-only view of the plan step S2-S3 built for an input
 * (no CUDA call).  For each generator matrix j < n_gamma_built: a[j] units
 * with three representatives, b[j] with one, f[j] free rows; order[0..n_used)
 * lists the matrices that are enumerated.  d_est is the random-code estimate
 * used to choose them; u0 the lightest representative.
 */
typedef struct {
    int32_t n_gamma_built, n_gamma_used, k_eff, s_rank, d_est, u0;
    int32_t order[16];
    int32_t a[16], b[16], f[16];
} dist_plan_info;
int dist_plan_info_get(const uint8_t *generator, int n, int K, int field, int n_stab,
                       dist_plan_info *info);

/*
 * dist_plan_unit -- host-only: representative `rep` of unit `unit` of
 * generator matrix `gamma` (units 0..a-1 first, then the b single-
 * representative ones) as 2n bytes (x | z) in the input's qubit order, with
 * its pivot qubit (-1 for a free row) and kind (0 rank-2 package or F4 row,
 * 1 rank-1 package, 2 free row).  For tests of the diagonalization.
 */
int dist_plan_unit(const uint8_t *generator, int n, int K, int field, int gamma, int unit,
                   int rep, uint8_t *vec_out, int *qubit, int *kind);

/*
 * Qubit stabilizer codes (Section 2).  The classical stabilizer code S of an
 * [[n, k, d(Q)]] code lies in its symplectic dual N = S^{perp_s} (the
 * classical normalizer code, dimension n + k); d(Q) = wt_s(N minus S) for
 * k > 0 and wt_s(S) for k = 0.
 *
 * dist_normalizer -- host only: a normalizer matrix of the code.
 *   stabilizers: m rows x 2n bytes in {0,1} (x | z), generators of S in any
 *                number (dependent rows are dropped); 1 <= n <= 128.
 *   generator_out: room for 2n rows x 2n bytes; receives *K_out rows whose
 *                first *n_stab_out rows are a basis of S and the rest
 *                logical operators (K = n + k, n_stab = n - k); for k = 0, a
 *                basis of S and n_stab = 0.
 *   DIST_EINVAL if a byte is not 0/1 or two generators anticommute;
 *   DIST_EZERO if every row is zero.
 * dist_init_stabilizer -- dist_normalizer, then dist_init and
 *   dist_set_exclude with its rows: dist_solve then returns d(Q), with a
 *   witness in N minus S (a logical operator of weight d(Q)).
 */
int dist_normalizer(const uint8_t *stabilizers, int n, int m, uint8_t *generator_out, int *K_out,
                    int *n_stab_out);
int dist_init_stabilizer(dist_code **out, const uint8_t *stabilizers, int n, int m);

/*
 * dist_intpeak -- integer issue microbenchmark used as the roofline
 * denominator.  Runs a loop of `iters` iterations of the enumeration's
 * per-codeword instruction mix (2 LOP3, 1 POPC, half a 3-way min) on every SM and
 * reports codewords per second (mix_per_s) plus the rates of POPC alone
 * and LOP3 alone (operations per second) and the SM clock seen (MHz).
 */
typedef struct {
    double mix_per_s, popc_per_s, lop3_per_s, sm_mhz;
    int32_t sms, blocks;
} dist_intpeak_result;
int dist_intpeak(dist_intpeak_result *out, int iters, void *cuda_stream);

/*
 * dist_solve_noalloc -- dist_init + dist_solve + dist_free in one call that
 * allocates no device memory.  The paper has no counterpart: this exists for
 * callers that cannot call cudaMalloc (code running inside another
 * framework's memory pool or under a fixed device-memory budget, or paths
 * where an allocation may not block or fail).  Every byte of device scratch
 * (bound and witness slots, segment table, binomial rows, generator-matrix
 * tables) lives in one file-scope device array of DIST_NOALLOC_MAX_BYTES
 * bytes that every GPU loading the library holds until process exit.
 *   generator, n, K, field: as dist_init (host memory, copied).
 *   n_stab: as dist_set_exclude (0 = plain minimum).
 *   out: caller-allocated result, as dist_solve.
 *   cuda_stream: cudaStream_t as void*; NULL = the legacy default stream.
 * Returns DIST_ERANGE, before touching the device, if the code's tables do
 * not fit the array.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) and sets the kernel's shared-memory limit;
 * make that first call before any stream capture.  No cudaMalloc, cudaFree,
 * pinned-host allocation, stream or event creation happens; host-side
 * planning uses ordinary heap memory.  All calls share the array and each
 * clears what must start at zero, so calls whose GPU work overlaps (other
 * streams, other host threads) race: serialize them.  gpu_seconds in the
 * result is the kernels' own run time (no events are created).
 */
#define DIST_NOALLOC_MAX_BYTES 65536
int dist_solve_noalloc(const uint8_t *generator, int n, int K, int field, int n_stab,
                       dist_result *out, void *cuda_stream);

/* Library version string and device info (name, SM count) of the current device. */
const char *dist_version(void);
const char *dist_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif
