/*
 * oracle.c -- plain CPU oracle for the symplectic minimum distance.
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the CPU
 * baseline of bench.py.  It shares no code, header, table or helper with the
 * GPU library, and the library never calls it.
 *
 * Two independent computations of d = wt_s(C) (Section 2, definitions):
 *   1. oracle_bruteforce -- every codeword of C once (Gray-code order over the
 *      coefficient vectors of a basis), d = min popcount(x | z).
 *   2. oracle_bz -- Algorithm 3 (Saved_isometry, Section 2.4): every row
 *      (a, b) becomes (a, b, a + b) in F2^{3n}, whose Hamming weight is twice
 *      wt_s(a, b); the Hamming minimum distance d_H of that binary code is
 *      found with the plain Brouwer-Zimmermann algorithm of Section 2.1
 *      (upper bound U from codewords seen, lower bound L from several
 *      systematic generator matrices, stop when L >= U); d = d_H / 2.
 *
 * Everything is exact integer arithmetic on 64-bit words.  Speed is not a
 * goal beyond splitting the enumeration over POSIX threads.
 */
#define _GNU_SOURCE
#include "oracle.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#include <unistd.h>

#define MAXN 128              /* qubits */
#define MAXK 256              /* F2 rows after the F4 -> F2 view */
#define WMAX 6                /* 64-bit words of a 3n-bit row, 3*128/64 */
#define KWMAX (MAXK / 64)     /* 64-bit words of a coefficient vector */
#define MAXGAMMA 8

static double now_s(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

static int popc64(uint64_t v) { return __builtin_popcountll(v); }

static int get_bit(const uint64_t *v, int i) { return (int)((v[i >> 6] >> (i & 63)) & 1u); }
static void set_bit(uint64_t *v, int i) { v[i >> 6] |= (uint64_t)1 << (i & 63); }

static int resolve_threads(int threads) {
    if (threads > 0) return threads;
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    return c > 0 ? (int)c : 1;
}

/* ------------------------------------------------------------------------- */
/* Input: F2 rows (x | z), the F2 view of an F4 input, and a rank reduction.  */
/* ------------------------------------------------------------------------- */

typedef struct {
    int n;                 /* qubits */
    int k;                 /* rank = number of basis rows */
    int s;                 /* rank of span(first n_stab input rows); basis rows 0..s-1 span it */
    uint64_t x[MAXK][2];   /* basis rows, x plane (n <= 128 bits) */
    uint64_t z[MAXK][2];   /* basis rows, z plane */
} f2_basis;

/* Reads the input, forms its F2 view and keeps, in input order, every row that
 * is independent of the rows kept before it.  Section 2.2 asks for linearly
 * independent rows; a dependent input is reduced rather than rejected. */
static int load_basis(const uint8_t *gen, int n, int K, int field, int n_stab, f2_basis *B) {
    if (!gen || n < 1 || n > MAXN || K < 0) return ORACLE_EINVAL;
    if (field != 2 && field != 4) return ORACLE_EINVAL;
    int rows = (field == 2) ? K : 2 * K;
    if (rows > MAXK) return ORACLE_EINVAL;
    if (n_stab < 0 || n_stab > K) return ORACLE_EINVAL;
    int stab_rows = (field == 2) ? n_stab : 2 * n_stab;

    uint64_t vx[MAXK][2], vz[MAXK][2];
    memset(vx, 0, sizeof vx);
    memset(vz, 0, sizeof vz);
    for (int r = 0; r < K; r++) {
        for (int i = 0; i < n; i++) {
            if (field == 2) {
                uint8_t a = gen[(size_t)r * 2 * n + i], b = gen[(size_t)r * 2 * n + n + i];
                if (a > 1 || b > 1) return ORACLE_EINVAL;
                if (a) set_bit(vx[r], i);
                if (b) set_bit(vz[r], i);
            } else {
                uint8_t v = gen[(size_t)r * n + i];
                if (v > 3) return ORACLE_EINVAL;
                int a = v & 1, b = (v >> 1) & 1;
                /* row g = a + alpha b */
                if (a) set_bit(vx[2 * r], i);
                if (b) set_bit(vz[2 * r], i);
                /* row alpha*g = a alpha + b alpha^2 = b + (a + b) alpha */
                if (b) set_bit(vx[2 * r + 1], i);
                if (a ^ b) set_bit(vz[2 * r + 1], i);
            }
        }
    }

    /* Echelon copy used only to test independence. */
    uint64_t ex[MAXK][4];
    int epiv[MAXK];
    int ne = 0;
    B->n = n;
    B->k = 0;
    B->s = 0;
    for (int r = 0; r < rows; r++) {
        uint64_t t[4] = {vx[r][0], vx[r][1], vz[r][0], vz[r][1]};
        for (int e = 0; e < ne; e++)
            if (get_bit(t, epiv[e]))
                for (int w = 0; w < 4; w++) t[w] ^= ex[e][w];
        int p = -1;
        for (int b = 0; b < 256 && p < 0; b++)
            if (get_bit(t, b)) p = b;
        if (p < 0) continue; /* dependent on the rows kept so far */
        memcpy(ex[ne], t, sizeof t);
        epiv[ne] = p;
        ne++;
        B->x[B->k][0] = vx[r][0];
        B->x[B->k][1] = vx[r][1];
        B->z[B->k][0] = vz[r][0];
        B->z[B->k][1] = vz[r][1];
        B->k++;
        if (r < stab_rows) B->s++;
    }
    return ORACLE_OK;
}

/* popcount(x | z): the symplectic weight of Section 2. */
static int wt_s(const uint64_t *x, const uint64_t *z) {
    return popc64(x[0] | z[0]) + popc64(x[1] | z[1]);
}

static void write_witness(uint8_t *witness, int n, const uint64_t *x, const uint64_t *z) {
    if (!witness) return;
    for (int i = 0; i < n; i++) {
        witness[i] = (uint8_t)get_bit(x, i);
        witness[n + i] = (uint8_t)get_bit(z, i);
    }
}

/* ------------------------------------------------------------------------- */
/* 1. Brute force.                                                           */
/* ------------------------------------------------------------------------- */

typedef struct {
    const f2_basis *B;
    uint64_t lo, hi;      /* coefficient-vector indices [lo, hi) of the Gray walk */
    int best_w;
    uint64_t best_k;
    uint64_t wdist[MAXN + 1];
} bf_job;

static void *bf_worker(void *arg) {
    bf_job *J = (bf_job *)arg;
    const f2_basis *B = J->B;
    uint64_t cx[2] = {0, 0}, cz[2] = {0, 0};
    uint64_t g = J->lo ^ (J->lo >> 1);
    for (int b = 0; b < B->k; b++)
        if ((g >> b) & 1u) {
            cx[0] ^= B->x[b][0]; cx[1] ^= B->x[b][1];
            cz[0] ^= B->z[b][0]; cz[1] ^= B->z[b][1];
        }
    J->best_w = 1 << 30;
    J->best_k = 0;
    for (uint64_t k = J->lo; k < J->hi; k++) {
        if (k != J->lo) {
            int b = __builtin_ctzll(k); /* Gray code: step k flips coefficient ctz(k) */
            cx[0] ^= B->x[b][0]; cx[1] ^= B->x[b][1];
            cz[0] ^= B->z[b][0]; cz[1] ^= B->z[b][1];
        }
        int w = wt_s(cx, cz);
        J->wdist[w]++;
        if (k == 0) continue; /* the zero codeword */
        uint64_t coeff = k ^ (k >> 1);
        if ((coeff >> B->s) == 0) continue; /* lies in S = span(first n_stab rows) */
        if (w < J->best_w) {
            J->best_w = w;
            J->best_k = k;
        }
    }
    return NULL;
}

int oracle_bruteforce(const uint8_t *gen, int n, int K, int field, int n_stab, int threads,
                      int *d_out, uint8_t *witness, uint64_t *wdist) {
    f2_basis B;
    int rc = load_basis(gen, n, K, field, n_stab, &B);
    if (rc) return rc;
    if (B.k > 40) return ORACLE_EINVAL;
    if (B.k == 0 || B.s == B.k) return ORACLE_EZERO;
    int T = resolve_threads(threads);
    uint64_t total = (uint64_t)1 << B.k;
    if ((uint64_t)T > total) T = (int)total;
    bf_job *jobs = (bf_job *)calloc((size_t)T, sizeof(bf_job));
    pthread_t *tid = (pthread_t *)calloc((size_t)T, sizeof(pthread_t));
    if (!jobs || !tid) { free(jobs); free(tid); return ORACLE_EINVAL; }
    for (int t = 0; t < T; t++) {
        jobs[t].B = &B;
        jobs[t].lo = total * (uint64_t)t / (uint64_t)T;
        jobs[t].hi = total * (uint64_t)(t + 1) / (uint64_t)T;
        pthread_create(&tid[t], NULL, bf_worker, &jobs[t]);
    }
    int best_w = 1 << 30;
    uint64_t best_k = 0;
    for (int t = 0; t < T; t++) {
        pthread_join(tid[t], NULL);
        if (jobs[t].best_w < best_w) {
            best_w = jobs[t].best_w;
            best_k = jobs[t].best_k;
        }
        if (wdist)
            for (int w = 0; w <= n; w++) wdist[w] += jobs[t].wdist[w];
    }
    free(jobs);
    free(tid);
    *d_out = best_w;
    if (witness) {
        uint64_t g = best_k ^ (best_k >> 1), cx[2] = {0, 0}, cz[2] = {0, 0};
        for (int b = 0; b < B.k; b++)
            if ((g >> b) & 1u) {
                cx[0] ^= B.x[b][0]; cx[1] ^= B.x[b][1];
                cz[0] ^= B.z[b][0]; cz[1] ^= B.z[b][1];
            }
        write_witness(witness, n, cx, cz);
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------- */
/* 2. Algorithm 3: isometry + plain Brouwer-Zimmermann (Hamming weight).     */
/* ------------------------------------------------------------------------- */

/* Row of F2^{3n}: bits [0,n) = a, [n,2n) = b, [2n,3n) = a + b. */
static void iso_row(const uint64_t *x, const uint64_t *z, int n, uint64_t *out) {
    memset(out, 0, WMAX * sizeof(uint64_t));
    for (int i = 0; i < n; i++) {
        int a = get_bit(x, i), b = get_bit(z, i);
        if (a) set_bit(out, i);
        if (b) set_bit(out, n + i);
        if (a ^ b) set_bit(out, 2 * n + i);
    }
}

int oracle_iso_weight(const uint8_t *row, int n) {
    if (!row || n < 1 || n > MAXN) return -1;
    uint64_t x[2] = {0, 0}, z[2] = {0, 0}, v[WMAX];
    for (int i = 0; i < n; i++) {
        if (row[i]) set_bit(x, i);
        if (row[n + i]) set_bit(z, i);
    }
    iso_row(x, z, n, v);
    int w = 0;
    for (int i = 0; i < WMAX; i++) w += popc64(v[i]);
    return w;
}

/* One systematic generator matrix Gamma_j of the isometry code: k rows in
 * reduced echelon form on its information set (pivot columns), with each
 * row's coefficient vector over the basis. */
typedef struct {
    int k;                       /* rank on the columns it was allowed to use */
    int f;                       /* rows without a pivot: K - k */
    uint64_t row[MAXK][WMAX];
    uint64_t coef[MAXK][KWMAX];
} gamma_mat;

typedef struct {
    const gamma_mat *G;
    int K, r, s, w3;
    /* jobs: (s0, s1) prefixes in lexicographic order, or a single job for r = 1 */
    int njobs;
    volatile int next;
    volatile int stop;
    double deadline;  /* absolute time, 0 = none */
    pthread_mutex_t mu;
    /* results merged under mu */
    int best_w;
    uint64_t best_c[WMAX];
    uint64_t codewords;
} bz_step;

static int hamming(const uint64_t *v, int w3) {
    int w = 0;
    for (int i = 0; i < w3; i++) w += popc64(v[i]);
    return w;
}

/* Is the codeword with these row indices outside S?  Its coefficient vector
 * over the basis must have a nonzero bit at a position >= s. */
static int outside_S(const gamma_mat *G, const int *idx, int r, int s, int K) {
    if (s == 0) return 1;
    uint64_t c[KWMAX] = {0};
    for (int t = 0; t < r; t++)
        for (int w = 0; w < KWMAX; w++) c[w] ^= G->coef[idx[t]][w];
    for (int b = s; b < K; b++)
        if (get_bit(c, b)) return 1;
    return 0;
}

static void decode_job(int j, int K, int *s0, int *s1) {
    /* jobs enumerate pairs s0 < s1 in lexicographic order */
    int a = 0;
    while (j >= K - 1 - a) {
        j -= K - 1 - a;
        a++;
    }
    *s0 = a;
    *s1 = a + 1 + j;
}

static void *bz_worker(void *arg) {
    bz_step *S = (bz_step *)arg;
    const gamma_mat *G = S->G;
    const int K = S->K, r = S->r, w3 = S->w3;
    int idx[MAXK];
    uint64_t acc[MAXK + 1][WMAX];
    int best_w = 1 << 30;
    uint64_t best_c[WMAX] = {0};
    uint64_t count = 0, since_check = 0;

    for (;;) {
        if (S->stop) break;
        int j = __sync_fetch_and_add(&S->next, 1);
        if (j >= S->njobs) break;
        memset(acc[0], 0, sizeof acc[0]);
        int level; /* number of fixed leading indices */
        if (r == 1) {
            /* single job: every row */
            for (int a = 0; a < K; a++) {
                count++;
                int w = hamming(G->row[a], w3);
                idx[0] = a;
                if (w < best_w && outside_S(G, idx, 1, S->s, K)) {
                    best_w = w;
                    memcpy(best_c, G->row[a], sizeof best_c);
                }
            }
            continue;
        }
        int s0, s1;
        decode_job(j, K, &s0, &s1);
        if (s1 > K - (r - 1)) continue; /* no room for the remaining r-2 indices */
        idx[0] = s0;
        idx[1] = s1;
        for (int w = 0; w < w3; w++) {
            acc[1][w] = G->row[s0][w];
            acc[2][w] = acc[1][w] ^ G->row[s1][w];
        }
        level = 2;
        if (r == 2) {
            count++;
            int w = hamming(acc[2], w3);
            if (w < best_w && outside_S(G, idx, 2, S->s, K)) {
                best_w = w;
                memcpy(best_c, acc[2], sizeof best_c);
            }
            continue;
        }
        /* Depth-first walk over idx[2..r-1] with idx increasing; acc[t+1] is
         * the sum of the rows idx[0..t]. */
        idx[level] = idx[level - 1];
        while (level >= 2) {
            idx[level]++;
            if (idx[level] > K - (r - level)) {
                level--;
                continue;
            }
            for (int w = 0; w < w3; w++) acc[level + 1][w] = acc[level][w] ^ G->row[idx[level]][w];
            if (level + 1 < r) {
                level++;
                idx[level] = idx[level - 1];
                continue;
            }
            count++;
            int wt = hamming(acc[r], w3);
            if (wt < best_w && outside_S(G, idx, r, S->s, K)) {
                best_w = wt;
                memcpy(best_c, acc[r], sizeof best_c);
            }
            if (++since_check >= (1u << 22)) {
                since_check = 0;
                if (S->stop) break;
                if (S->deadline > 0 && now_s() > S->deadline) {
                    S->stop = 1;
                    break;
                }
            }
        }
    }
    pthread_mutex_lock(&S->mu);
    S->codewords += count;
    if (best_w < S->best_w) {
        S->best_w = best_w;
        memcpy(S->best_c, best_c, sizeof best_c);
    }
    pthread_mutex_unlock(&S->mu);
    return NULL;
}

/* Builds Gamma_j: reduced echelon form of the basis using only columns not
 * used by Gamma_1 .. Gamma_{j-1}; returns its rank. */
static int build_gamma(const uint64_t (*base)[WMAX], int K, int ncols, const uint8_t *used,
                       gamma_mat *G, uint8_t *pivot_of_this) {
    memset(pivot_of_this, 0, (size_t)ncols);
    for (int i = 0; i < K; i++) {
        memcpy(G->row[i], base[i], sizeof G->row[i]);
        memset(G->coef[i], 0, sizeof G->coef[i]);
        set_bit(G->coef[i], i);
    }
    int row = 0;
    for (int col = 0; col < ncols && row < K; col++) {
        if (used[col]) continue;
        int p = -1;
        for (int i = row; i < K; i++)
            if (get_bit(G->row[i], col)) { p = i; break; }
        if (p < 0) continue;
        if (p != row) {
            uint64_t t[WMAX], c[KWMAX];
            memcpy(t, G->row[p], sizeof t); memcpy(G->row[p], G->row[row], sizeof t); memcpy(G->row[row], t, sizeof t);
            memcpy(c, G->coef[p], sizeof c); memcpy(G->coef[p], G->coef[row], sizeof c); memcpy(G->coef[row], c, sizeof c);
        }
        for (int i = 0; i < K; i++)
            if (i != row && get_bit(G->row[i], col)) {
                for (int w = 0; w < WMAX; w++) G->row[i][w] ^= G->row[row][w];
                for (int w = 0; w < KWMAX; w++) G->coef[i][w] ^= G->coef[row][w];
            }
        pivot_of_this[col] = 1;
        row++;
    }
    G->k = row;
    G->f = K - row;
    return row;
}

int oracle_bz(const uint8_t *gen, int n, int K, int field, int n_stab, int threads,
              double time_budget, oracle_result *res, uint8_t *witness,
              int32_t *ltrace, int ltrace_cap, int *ltrace_len) {
    if (!res) return ORACLE_EINVAL;
    memset(res, 0, sizeof *res);
    if (ltrace_len) *ltrace_len = 0;
    f2_basis B;
    int rc = load_basis(gen, n, K, field, n_stab, &B);
    if (rc) return rc;
    res->k_eff = B.k;
    if (B.k == 0 || B.s == B.k) return ORACLE_EZERO;
    const int Kb = B.k, ncols = 3 * n, w3 = (ncols + 63) / 64;
    int T = resolve_threads(threads);
    res->threads = T;

    /* Algorithm 3, first step: B := iso(A). */
    uint64_t (*base)[WMAX] = (uint64_t (*)[WMAX])calloc(MAXK, sizeof *base);
    gamma_mat *G = (gamma_mat *)calloc(MAXGAMMA, sizeof(gamma_mat));
    if (!base || !G) { free(base); free(G); return ORACLE_EINVAL; }
    for (int i = 0; i < Kb; i++) iso_row(B.x[i], B.z[i], n, base[i]);

    /* Systematic generator matrices on disjoint information sets, each on
     * the columns the earlier ones left unused, until no unused column has
     * positive rank.  Gamma_1 has full rank; a later Gamma_j of rank k_j < K
     * has f_j = K - k_j rows without a pivot, and the bound below counts it
     * with r + 1 - f_j (the lower bound of Algorithm 2 treats its second
     * matrix the same way). */
    uint8_t used[3 * MAXN], piv[3 * MAXN];
    memset(used, 0, sizeof used);
    int m = 0;
    while (m < MAXGAMMA) {
        int k = build_gamma((const uint64_t(*)[WMAX])base, Kb, ncols, used, &G[m], piv);
        if (k == 0) break;
        for (int c = 0; c < ncols; c++) used[c] |= piv[c];
        m++;
    }
    res->n_gamma = m;

    double t0 = now_s();
    double deadline = time_budget > 0 ? t0 + time_budget : 0.0;
    int U = 1 << 30;              /* upper bound on d_H */
    uint64_t best_c[WMAX] = {0};
    int L = 0;                    /* lower bound on d_H */
    for (int j = 0; j < m; j++) L += (1 - G[j].f > 0) ? 1 - G[j].f : 0;
    int nl = 0, complete = 0;
    uint64_t codewords = 0;

    for (int r = 1; r <= Kb && !complete; r++) {
        res->rounds = r;
        for (int j = 0; j < m; j++) {
            bz_step S;
            memset(&S, 0, sizeof S);
            S.G = &G[j];
            S.K = Kb;
            S.r = r;
            S.s = B.s;
            S.w3 = w3;
            S.njobs = (r == 1) ? 1 : Kb * (Kb - 1) / 2;
            S.deadline = deadline;
            S.best_w = 1 << 30;
            pthread_mutex_init(&S.mu, NULL);
            int TT = (r == 1) ? 1 : T;
            pthread_t tid[512];
            if (TT > 512) TT = 512;
            for (int t = 0; t < TT; t++) pthread_create(&tid[t], NULL, bz_worker, &S);
            for (int t = 0; t < TT; t++) pthread_join(tid[t], NULL);
            pthread_mutex_destroy(&S.mu);
            codewords += S.codewords;
            if (S.best_w < U) {
                U = S.best_w;
                memcpy(best_c, S.best_c, sizeof best_c);
            }
            if (S.stop) goto out; /* time budget exhausted inside this step */
            /* Gamma_1..Gamma_j have finished round r, the others round r-1:
             * every codeword not yet seen has at least r+1 (resp. r) nonzero
             * coefficients in each matrix, hence at least r+1-f (resp. r-f)
             * ones on that matrix's information set, and the sets are disjoint. */
            L = 0;
            for (int i = 0; i < m; i++) {
                int t = (i <= j ? r + 1 : r) - G[i].f;
                L += t > 0 ? t : 0;
            }
            if (ltrace && nl < ltrace_cap) ltrace[nl++] = L;
            if (L >= U) {
                complete = 1;
                break;
            }
        }
    }
out:
    free(base);
    free(G);
    res->seconds = now_s() - t0;
    res->codewords = codewords;
    res->complete = complete;
    if (ltrace_len) *ltrace_len = nl;
    if (U >= (1 << 30)) return complete ? ORACLE_EZERO : ORACLE_EINCOMPLETE;
    res->d = U / 2;
    res->lower = complete ? U / 2 : (L + 1) / 2;
    if (witness) {
        /* the first 2n bits of the isometry image are (a, b) */
        for (int i = 0; i < n; i++) {
            witness[i] = (uint8_t)get_bit(best_c, i);
            witness[n + i] = (uint8_t)get_bit(best_c, n + i);
        }
    }
    return complete ? ORACLE_OK : ORACLE_EINCOMPLETE;
}
