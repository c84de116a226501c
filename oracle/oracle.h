/*
 * oracle.h -- CPU oracle for the symplectic minimum distance.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library (paper_2408_10743_gb300/)
 * links, loads or calls this code.  It exists so that tests, the smoke check
 * and the CPU-baseline leg of bench.py can compare the GPU path with a plain,
 * slow, obviously correct implementation written independently from it.
 *
 * What it computes (Section 2, definitions of wt_s and wt_s(C)):
 *   d = min { wt_s(c) : c in C, c != 0 },   wt_s(a,b) = #{ i : a_i != 0 or b_i != 0 },
 * where C is the F2-span of the given rows of F2^{2n}.  An F4-linear input
 * (Section 2.3) is first replaced by its F2 view: every F4 row g contributes
 * the two F2 rows g and alpha*g, whose F2-span is the F4-span of the input.
 * With n_stab > 0 the minimum is taken over C minus span(first n_stab rows),
 * the check of the modified Brouwer-Zimmermann algorithm (Section 2.1).
 *
 * Two independent ways of computing d:
 *   oracle_bruteforce: Gray-code walk over every coefficient vector (tiny K).
 *   oracle_bz:         Algorithm 3 (Saved_isometry): map (a,b) -> (a,b,a+b),
 *                      plain binary Brouwer-Zimmermann for the Hamming weight
 *                      on several systematic generator matrices, d = d_H / 2.
 *
 * Input layout (same as the library's):
 *   field 2: K rows x 2n bytes in {0,1}: x_0..x_{n-1} | z_0..z_{n-1}.
 *   field 4: K rows x n bytes in {0,1,2,3}: v = a + 2b stands for a + alpha*b
 *            (x-plane a, z-plane b), alpha^2 = alpha + 1.
 * Limits: 1 <= n <= 128; K <= 256 F2 rows after the F4 -> F2 view.
 *
 * Return codes: 0 ok; -1 invalid argument; -6 the code (or C minus S) has no
 * nonzero codeword; -5 time budget exhausted before d was certified.
 */
#ifndef DIST_ORACLE_H
#define DIST_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_EINCOMPLETE (-5)
#define ORACLE_EZERO (-6)

/* Brute force over all 2^K' coefficient vectors of the F2 view (K' <= 40).
 *   d_out:    minimum symplectic weight of a nonzero codeword (outside S if n_stab > 0).
 *   witness:  2n bytes (x|z) of one codeword of weight d, or NULL.
 *   wdist:    n+1 counters, wdist[w] += #coefficient vectors (zero one included)
 *             whose codeword has weight w, or NULL.
 *   threads:  0 = all online cores. */
int oracle_bruteforce(const uint8_t *gen, int n, int K, int field, int n_stab,
                      int threads, int *d_out, uint8_t *witness, uint64_t *wdist);

typedef struct {
    int32_t d;          /* certified distance (upper bound U/2 when incomplete) */
    int32_t lower;      /* final lower bound on d (ceil(L/2)) */
    int32_t rounds;     /* last round r that was started */
    int32_t n_gamma;    /* number of systematic generator matrices used */
    int32_t k_eff;      /* rank of the input */
    int32_t complete;   /* 1 if d is certified */
    uint64_t codewords; /* r-subsets whose sum was formed */
    double seconds;     /* wall time of the enumeration */
    int32_t threads;    /* threads actually used */
    int32_t pad;
} oracle_result;

/* Algorithm 3 (Saved_isometry) with plain binary Brouwer-Zimmermann.
 *   time_budget: seconds (<= 0 means unlimited); when exceeded the call returns
 *                ORACLE_EINCOMPLETE with res->d = U/2 and res->lower set.
 *   witness:     2n bytes (x|z), or NULL.
 *   ltrace:      if not NULL, receives the Hamming-weight lower bound L after
 *                every (round, matrix) step, up to ltrace_cap entries; the
 *                number written is returned in *ltrace_len. */
int oracle_bz(const uint8_t *gen, int n, int K, int field, int n_stab, int threads,
              double time_budget, oracle_result *res, uint8_t *witness,
              int32_t *ltrace, int ltrace_cap, int *ltrace_len);

/* Hamming weight of the isometry image (a, b, a+b) of one F2 row (2n bytes).
 * Exposed so that tests can check the identity wt_H = 2 wt_s. */
int oracle_iso_weight(const uint8_t *row, int n);

#ifdef __cplusplus
}
#endif
#endif
