// walk.cuh -- what one lane of the enumeration kernel does (steps S4/S5).
//
// A lane owns a contiguous range of combination ranks inside one segment
// (i units from the A-units, r-i from the B-units) of round r of one
// generator matrix.  For every subset it evaluates every choice of
// representatives (F2: 3^i, F4: 3^(i-1) with the first unit's scalar fixed).
//
// Order of subsets: revolving-door Gray code (Knuth, TAOCP 4A, 7.2.1.3):
//   RD(n, t) = RD(n-1, t) followed by reversed RD(n-1, t-1) with n-1 added,
//   rank(c_t > ... > c_1) = C(c_t + 1, t) - 1 - rank(c_{t-1} > ... > c_1).
// Consecutive subsets differ by one unit out and one unit in; a lane unranks
// its first subset from the combinatorial number system and then steps.
//
// Order of representatives (the fast path, i >= 4 varying units).  Sorted
// positions of the subset play three roles:
//   i-1, i-2  : a 9-entry register table T of word-0 partial sums;
//   i-3, i-4  : two "register digits" B and A whose deltas sit in registers;
//   the rest  : "dynamic digits", advanced by a modular ternary Gray code
//               (step k changes digit nu_3(k) by +1 mod 3).
// Changing a digit from e to e+1 XORs the unit's third representative
// (rep0 ^ rep1 ^ rep2 = 0), so one block of 81 codewords is 9 table sweeps
// separated by the 8 steps of a 2-digit ternary Gray code over A and B, and
// a dynamic step follows every block.  A codeword costs two LOP3, one POPC
// and about half a 3-way min on word 0 of each plane.  Word 0 holds qubits
// that are not pivots of this generator matrix, so popc(word 0) is a sharp
// lower bound on the weight; only when a block's minimum falls below the
// current upper bound is it re-walked with full weights (the slow path), so
// the result is exact.
#pragma once
#include <math.h>

#include "dist_types.h"

namespace dist {

#if defined(__CUDACC__)
#define DIST_HD_COLD __host__ __device__ __noinline__
#if defined(DIST_FAST_NOINLINE)
#define DIST_HD_FAST __host__ __device__ __noinline__
#else
#define DIST_HD_FAST __host__ __device__ __forceinline__
#endif
#else
#define DIST_HD_COLD inline
#define DIST_HD_FAST inline
#endif

struct U2 {
    uint32_t x, z;
};

DIST_HD int popc32(uint32_t v) {
#if defined(__CUDA_ARCH__)
    return __popc(v);
#else
    return __builtin_popcount(v);
#endif
}

DIST_HD uint32_t min3u(uint32_t a, uint32_t b, uint32_t c) {
#if defined(__CUDA_ARCH__)
    return __vimin3_u32(a, b, c);
#else
    uint32_t m = a < b ? a : b;
    return m < c ? m : c;
#endif
}

DIST_HD unsigned long long binom_at(const unsigned long long* B, int stride, int n, int k) {
    if (k < 0 || n < k) return 0ull;
    return B[n * stride + k];
}

// The unranking estimate below needs only a few correct bits: the device
// takes the hardware log2 and reciprocal approximations for it.
#if defined(__CUDA_ARCH__)
#define DIST_EST_LOG2(x) __log2f(x)
#define DIST_EST_RCP(x) __fdividef(1.0f, (x))
#else
#define DIST_EST_LOG2(x) log2f(x)
#define DIST_EST_RCP(x) (1.0f / (x))
#endif

// Largest c in [lo, hi] with C(c, t) <= R (C(lo, t) <= R holds); C(c + 1, t)
// goes to *next.  The start is the closed-form estimate C(c, t) ~
// (c - (t-1)/2)^t / t!, i.e. c ~ (R t!)^(1/t) + (t-1)/2, with lgf = log2(t!);
// exact binomial lookups then move it to the answer, so the result does not
// depend on the rounding of the estimate.  C(c, t) and C(c + 1, t) are read
// together, so an estimate that is already right costs one round trip to the
// table, and C(c + 1, t) is the value the caller needs next.
DIST_HD int cns_top(const unsigned long long* B, int stride, int t, unsigned long long R, int lo, int hi,
                    float lgf, unsigned long long* next) {
    if (t == 1) {  // C(c, 1) = c
        const int c = (int)(R < (unsigned long long)hi ? R : (unsigned long long)hi);
        *next = (unsigned long long)c + 1ull;
        return c;
    }
    const float x =
        exp2f((DIST_EST_LOG2((float)R + 0.5f) + lgf) * DIST_EST_RCP((float)t)) + 0.5f * (float)(t - 1);
    int c = x < (float)lo ? lo : (x > (float)hi ? hi : (int)x);
    unsigned long long b0 = binom_at(B, stride, c, t), b1 = binom_at(B, stride, c + 1, t);
    while (c > lo && b0 > R) {
        --c;
        b1 = b0;
        b0 = binom_at(B, stride, c, t);
    }
    while (c < hi && b1 <= R) {
        ++c;
        b0 = b1;
        b1 = binom_at(B, stride, c + 1, t);
    }
    *next = b1;
    return c;
}

// Subset of revolving-door rank R (0 <= R < C(n, t)), t elements of
// {0..n-1}, written ascending into s: the largest element c_t is the largest
// c with C(c, t) <= R, and the rest is the subset of rank C(c_t + 1, t) - 1 - R
// of {0..c_t - 1}.
DIST_HD void rd_unrank(const unsigned long long* B, int stride, int n, unsigned long long R, int t,
                       uint8_t* s) {
    float lgf = 0.0f;  // log2(tt!) for the estimate
    for (int k = 2; k <= t; k++) lgf += DIST_EST_LOG2((float)k);
    for (int tt = t; tt >= 1; --tt) {
        unsigned long long nx;
        const int c = cns_top(B, stride, tt, R, tt - 1, n - 1, lgf, &nx);
        s[tt - 1] = (uint8_t)c;
        R = nx - 1 - R;
        n = c;
        lgf -= DIST_EST_LOG2((float)tt);
    }
}

// Successor in revolving-door order (Knuth's Algorithm R, steps R3-R5) of
// the ascending t-subset s of {0..n-1}.  The caller never steps past the last.
DIST_HD void rd_next(uint8_t* s, int t, int n) {
#define DIST_CJ(j) ((j) <= t ? (int)s[(j)-1] : n)
    int j;
    if (t & 1) {
        if (s[0] + 1 < DIST_CJ(2)) {
            s[0]++;
            return;
        }
        j = 2;
        goto r4;
    } else {
        if (s[0] > 0) {
            s[0]--;
            return;
        }
        j = 2;
        goto r5;
    }
r4:
    if (j > t) return;
    if (DIST_CJ(j) >= j) {
        s[j - 1] = s[j - 2];
        s[j - 2] = (uint8_t)(j - 2);
        return;
    }
    j++;
r5:
    if (j > t) return;
    if (DIST_CJ(j) + 1 < DIST_CJ(j + 1)) {
        s[j - 2] = s[j - 1];
        s[j - 1]++;
        return;
    }
    j++;
    goto r4;
#undef DIST_CJ
}

// What a lane reads for one segment.  reps / r0 / binom live in shared
// memory on the device.
struct LaneCtx {
    const uint32_t* reps;              // [u][3][2][W]
    const U2* r0;                      // [a][3]: word 0 of the A-units' representatives
    const U2* r1;                      // [a][3]: word 1 (W >= 2)
    const uint32_t* flags;             // [u]: bit 0 / bit 1: package with pivot beyond word 0 / 1
    const uint32_t* coefs;             // [u][3][2][CW]
    const unsigned long long* binom;   // [rows][bstride]
    const uint32_t* outside;
    int bstride;
    int a, b, W, CW, gamma, proj, exclude;
    int t1;                            // two-word filter when thr - P exceeds this
    uint32_t a_all;                    // AND of the A-units' flags: bit set = every A-unit has it
};

DIST_HD const uint32_t* rep_ptr(const LaneCtx& C, int unit, int e, int plane) {
    return C.reps + ((unit * 3 + e) * 2 + plane) * C.W;
}

// Exact weight of the combination (A-units sA with digits eA, B-units sB);
// records it when it beats thr and, in exclusion mode, lies outside S.
// Returns the new threshold.  consider() and block_slow() are inlined: as
// called functions they made the compiler keep more of the fast loop's state
// on the stack around their call sites.  The functions that stay calls take
// the sink and the threshold by value: an address passed to a function that
// is not inlined would keep the caller's copy in local memory through its
// hot loop.
template <class Sink>
DIST_HD_FAST uint32_t consider(const LaneCtx& C, Sink sink, uint32_t thr, int i, const uint8_t* sA,
                               const uint8_t* eA, int nb, const uint8_t* sB) {
    uint32_t x[DIST_MAXW], z[DIST_MAXW];
    for (int w = 0; w < DIST_MAXW; w++) x[w] = z[w] = 0;
    for (int p = 0; p < i; p++) {
        const uint32_t* rx = rep_ptr(C, sA[p], eA[p], 0);
        const uint32_t* rz = rep_ptr(C, sA[p], eA[p], 1);
        for (int w = 0; w < C.W; w++) {
            x[w] ^= rx[w];
            z[w] ^= rz[w];
        }
    }
    for (int q = 0; q < nb; q++) {
        const uint32_t* rx = rep_ptr(C, C.a + sB[q], 0, 0);
        const uint32_t* rz = rep_ptr(C, C.a + sB[q], 0, 1);
        for (int w = 0; w < C.W; w++) {
            x[w] ^= rx[w];
            z[w] ^= rz[w];
        }
    }
    uint32_t wt = 0;
    for (int w = 0; w < C.W; w++) wt += popc32(x[w] | z[w]);
    if (wt >= thr) return thr;
    if (C.exclude) {
        uint32_t acc = 0;
        for (int w = 0; w < C.CW; w++) {
            uint32_t c0 = 0, c1 = 0;
            for (int p = 0; p < i; p++) {
                const uint32_t* cp = C.coefs + ((sA[p] * 3 + eA[p]) * 2) * C.CW;
                c0 ^= cp[w];
                c1 ^= cp[C.CW + w];
            }
            for (int q = 0; q < nb; q++) {
                const uint32_t* cp = C.coefs + (((C.a + sB[q]) * 3) * 2) * C.CW;
                c0 ^= cp[w];
                c1 ^= cp[C.CW + w];
            }
            acc |= (c0 | c1) & C.outside[w];
        }
        if (!acc) return thr;  // inside S = span(first n_stab rows)
    }
    uint8_t units[DIST_MAXR], digits[DIST_MAXR];
    for (int p = 0; p < i; p++) {
        units[p] = sA[p];
        digits[p] = eA[p];
    }
    for (int q = 0; q < nb; q++) {
        units[i + q] = (uint8_t)(C.a + sB[q]);
        digits[i + q] = 0;
    }
    sink.record(wt, C.gamma, i + nb, units, digits);
    return wt;
}

// Every representative choice of one subset, each weighed on all W words
// (small i, where the fast path's table does not apply).  The sum starts with
// every unit at representative 0 and then follows a modular ternary Gray
// code over the free digits: the digit that changes is the first one of a
// ternary counter that does not wrap, and changing digit p from e to e+1
// XORs the unit's representative (e+2) mod 3.  The sum stays in registers;
// consider() re-weighs and records only a combination lighter than thr.
template <int W, class Sink>
DIST_HD void eval_generic_w(const LaneCtx& C, Sink& sink, uint32_t& thr, int i, const uint8_t* sA,
                            int nb, const uint8_t* sB) {
    uint32_t x[W], z[W];
#pragma unroll
    for (int w = 0; w < W; w++) x[w] = z[w] = 0;
    for (int p = 0; p < i; p++) {
        const uint32_t* r = C.reps + (sA[p] * 3) * 2 * W;
#pragma unroll
        for (int w = 0; w < W; w++) {
            x[w] ^= r[w];
            z[w] ^= r[W + w];
        }
    }
    for (int q = 0; q < nb; q++) {
        const uint32_t* r = C.reps + ((C.a + sB[q]) * 3) * 2 * W;
#pragma unroll
        for (int w = 0; w < W; w++) {
            x[w] ^= r[w];
            z[w] ^= r[W + w];
        }
    }
    uint8_t e[DIST_MAXR], cnt[DIST_MAXR];
    for (int p = 0; p < i; p++) e[p] = cnt[p] = 0;
    const int first = C.proj ? 1 : 0;
    const int nd = i - first;
    for (;;) {
        uint32_t wt = 0;
#pragma unroll
        for (int w = 0; w < W; w++) wt += (uint32_t)popc32(x[w] | z[w]);
        if (wt < thr) thr = consider(C, sink, thr, i, sA, e, nb, sB);
        int q = 0;
        while (q < nd && cnt[q] == 2) {
            cnt[q] = 0;
            ++q;
        }
        if (q >= nd) break;
        ++cnt[q];
        const int p = first + q;
        const int ee = e[p];
        const uint32_t* r = C.reps + (sA[p] * 3 + (ee == 0 ? 2 : ee - 1)) * 2 * W;
#pragma unroll
        for (int w = 0; w < W; w++) {
            x[w] ^= r[w];
            z[w] ^= r[W + w];
        }
        e[p] = (uint8_t)(ee == 2 ? 0 : ee + 1);
    }
}

template <class Sink>
DIST_HD_COLD uint32_t eval_generic(const LaneCtx& C, Sink sink, uint32_t thr, int i, const uint8_t* sA,
                                   int nb, const uint8_t* sB) {
    switch (C.W) {
        case 1: eval_generic_w<1>(C, sink, thr, i, sA, nb, sB); break;
        case 2: eval_generic_w<2>(C, sink, thr, i, sA, nb, sB); break;
        case 3: eval_generic_w<3>(C, sink, thr, i, sA, nb, sB); break;
        default: eval_generic_w<4>(C, sink, thr, i, sA, nb, sB); break;
    }
    return thr;
}

// Slow path of one 81-codeword block: each codeword whose lower bound
// (popcount of its first F words + P) is below thr is weighed in full.
// (vbx, vbz) holds the first F words of the B-units' sum; eB0 is digit B's
// value at the block start (digit A starts every block at 0); P counts the
// subset's packages whose pivot lies beyond the first F words, each worth one
// more unit of weight.
template <int F, class Sink>
DIST_HD_FAST uint32_t block_slow(const LaneCtx& C, Sink sink, uint32_t thr, int i, const uint8_t* sA,
                                 const uint8_t* dig, int nb, const uint8_t* sB, uint32_t vbx0, uint32_t vbx1,
                                 uint32_t vbz0, uint32_t vbz1, int eB0, uint32_t P) {
    const uint32_t vbx[2] = {vbx0, vbx1}, vbz[2] = {vbz0, vbz1};
    uint8_t e[DIST_MAXR];
    const U2* tab[2] = {C.r0, C.r1};
    uint32_t bx[F], bz[F];
    for (int f = 0; f < F; f++) {
        bx[f] = vbx[f];
        bz[f] = vbz[f];
    }
    for (int p = 0; p < i - 4; p++) {
        e[p] = dig[p];
        for (int f = 0; f < F; f++) {
            const U2 v = tab[f][sA[p] * 3 + dig[p]];
            bx[f] ^= v.x;
            bz[f] ^= v.z;
        }
    }
    for (int kk = 0; kk < 9; kk++) {
        const int eA = (kk - kk / 3) % 3;
        const int eB = (eB0 + kk / 3) % 3;
        for (int j = 0; j < 9; j++) {
            const int e0 = j % 3, e1 = j / 3;
            uint32_t lb = P;
            for (int f = 0; f < F; f++) {
                const U2* ra = tab[f] + sA[i - 4] * 3;
                const U2* rb = tab[f] + sA[i - 3] * 3;
                const U2* r0 = tab[f] + sA[i - 2] * 3;
                const U2* r1 = tab[f] + sA[i - 1] * 3;
                const uint32_t tx = bx[f] ^ ra[eA].x ^ rb[eB].x ^ r0[e0].x ^ r1[e1].x;
                const uint32_t tz = bz[f] ^ ra[eA].z ^ rb[eB].z ^ r0[e0].z ^ r1[e1].z;
                lb += (uint32_t)popc32(tx | tz);
            }
            if (lb >= thr) continue;
            e[i - 4] = (uint8_t)eA;
            e[i - 3] = (uint8_t)eB;
            e[i - 2] = (uint8_t)e0;
            e[i - 1] = (uint8_t)e1;
            thr = consider(C, sink, thr, i, sA, e, nb, sB);
        }
    }
    return thr;
}

// Popcount of codeword j of the current base (first F words).
template <int F>
DIST_HD uint32_t word_weight(const uint32_t (&bx)[F], const uint32_t (&bz)[F], const uint32_t (&Tx)[F][9],
                             const uint32_t (&Tz)[F][9], int j) {
    uint32_t c = 0;
#pragma unroll
    for (int f = 0; f < F; f++) c += (uint32_t)popc32((bx[f] ^ Tx[f][j]) | (bz[f] ^ Tz[f][j]));
    return c;
}

// Fast path: subsets with at least four varying units, filter on the first
// F words of each plane (F = 1, or 2 when the bound is still far above the
// distance).  Kept in one function so that only its own state (table,
// register-digit deltas, base words, counters) is live in the inner loop.
template <int F, class Sink>
DIST_HD_FAST void eval_fast(const LaneCtx& C, Sink& sink, uint32_t& thr, int i, const uint8_t* sA,
                            uint8_t* dig, int nb, const uint8_t* sB, const uint32_t* vbx,
                            const uint32_t* vbz, uint32_t P) {
    const U2* tab[2] = {C.r0, C.r1};
    uint32_t Tx[F][9], Tz[F][9];
    U2 Da0[F], Da1[F], Da2[F], Db0[F], Db1[F], Db2[F];
    uint32_t bx[F], bz[F];
#pragma unroll
    for (int f = 0; f < F; f++) {
        const U2* r0 = tab[f] + sA[i - 2] * 3;
        const U2* r1 = tab[f] + sA[i - 1] * 3;
        const U2 a0 = r0[0], a1 = r0[1], a2 = r0[2], b0 = r1[0], b1 = r1[1], b2 = r1[2];
        Tx[f][0] = a0.x ^ b0.x; Tz[f][0] = a0.z ^ b0.z;
        Tx[f][1] = a1.x ^ b0.x; Tz[f][1] = a1.z ^ b0.z;
        Tx[f][2] = a2.x ^ b0.x; Tz[f][2] = a2.z ^ b0.z;
        Tx[f][3] = a0.x ^ b1.x; Tz[f][3] = a0.z ^ b1.z;
        Tx[f][4] = a1.x ^ b1.x; Tz[f][4] = a1.z ^ b1.z;
        Tx[f][5] = a2.x ^ b1.x; Tz[f][5] = a2.z ^ b1.z;
        Tx[f][6] = a0.x ^ b2.x; Tz[f][6] = a0.z ^ b2.z;
        Tx[f][7] = a1.x ^ b2.x; Tz[f][7] = a1.z ^ b2.z;
        Tx[f][8] = a2.x ^ b2.x; Tz[f][8] = a2.z ^ b2.z;
        // digit A starts every block at 0; its deltas for e -> e+1 are rep[(e+2)%3]
        const U2* ra = tab[f] + sA[i - 4] * 3;
        const U2* rb = tab[f] + sA[i - 3] * 3;
        Da0[f] = ra[2]; Da1[f] = ra[0]; Da2[f] = ra[1];
        Db0[f] = rb[2]; Db1[f] = rb[0]; Db2[f] = rb[1];
        bx[f] = vbx[f] ^ ra[0].x ^ rb[0].x;
        bz[f] = vbz[f] ^ ra[0].z ^ rb[0].z;
        for (int p = 0; p < i - 4; p++) {
            const U2 v = tab[f][sA[p] * 3 + dig[p]];
            bx[f] ^= v.x;
            bz[f] ^= v.z;
        }
    }
    int eB = 0;
    const int first = C.proj ? 1 : 0;
    const int nd = i - 4 - first;
    uint32_t nk = 1;
    for (int q = 0; q < nd; q++) nk *= 3u;
    for (uint32_t k = 0; k < nk; ++k) {
        if (k) {
            uint32_t kk = k;
            int q = 0;
            while (kk % 3u == 0u) {
                kk /= 3u;
                ++q;
            }
            const int p = first + q;
            const int e = dig[p];
#pragma unroll
            for (int f = 0; f < F; f++) {
                const U2 v = tab[f][sA[p] * 3 + (e == 0 ? 2 : e - 1)];
                bx[f] ^= v.x;
                bz[f] ^= v.z;
            }
            dig[p] = (uint8_t)(e == 2 ? 0 : e + 1);
        }
        uint32_t m = 0xFFFFu;
#define DIST_SWEEP9()                                                                         \
    do {                                                                                      \
        const uint32_t c0 = word_weight<F>(bx, bz, Tx, Tz, 0), c1 = word_weight<F>(bx, bz, Tx, Tz, 1); \
        const uint32_t c2 = word_weight<F>(bx, bz, Tx, Tz, 2), c3 = word_weight<F>(bx, bz, Tx, Tz, 3); \
        const uint32_t c4 = word_weight<F>(bx, bz, Tx, Tz, 4), c5 = word_weight<F>(bx, bz, Tx, Tz, 5); \
        const uint32_t c6 = word_weight<F>(bx, bz, Tx, Tz, 6), c7 = word_weight<F>(bx, bz, Tx, Tz, 7); \
        const uint32_t c8 = word_weight<F>(bx, bz, Tx, Tz, 8);                               \
        m = min3u(m, min3u(c0, c1, c2), min3u(c3, c4, c5));                                   \
        m = min3u(m, min3u(c6, c7, c8), m);                                                   \
    } while (0)
#define DIST_STEP(D)                          \
    do {                                      \
        _Pragma("unroll") for (int f = 0; f < F; f++) { \
            bx[f] ^= D[f].x;                  \
            bz[f] ^= D[f].z;                  \
        }                                     \
    } while (0)
        DIST_SWEEP9();
        DIST_STEP(Da0);
        DIST_SWEEP9();
        DIST_STEP(Da1);
        DIST_SWEEP9();
        DIST_STEP(Db0);
        DIST_SWEEP9();
        DIST_STEP(Da2);
        DIST_SWEEP9();
        DIST_STEP(Da0);
        DIST_SWEEP9();
        DIST_STEP(Db1);
        DIST_SWEEP9();
        DIST_STEP(Da1);
        DIST_SWEEP9();
        DIST_STEP(Da2);
        DIST_SWEEP9();
#undef DIST_SWEEP9
#undef DIST_STEP
        // weight >= popcount(first F words) + P: only then can a codeword beat thr
        if (m + P < thr) thr = block_slow<F>(C, sink, thr, i, sA, dig, nb, sB, vbx[0], vbx[1], vbz[0], vbz[1], eB, P);
#pragma unroll
        for (int f = 0; f < F; f++) {  // B moved twice: rotate its delta triple by two
            const U2 t = Db2[f];
            Db2[f] = Db1[f];
            Db1[f] = Db0[f];
            Db0[f] = t;
        }
        eB = eB == 0 ? 2 : eB - 1;
    }
}

// First two words of the sum of the chosen B-units' single representatives,
// and how many of them are packages with a pivot beyond word 0 (P1) and
// beyond word 1 (P2).
DIST_HD void b_words(const LaneCtx& C, int nb, const uint8_t* sB, uint32_t* x, uint32_t* z,
                     uint32_t& P1, uint32_t& P2) {
    x[0] = z[0] = x[1] = z[1] = 0;
    P1 = P2 = 0;
    for (int q = 0; q < nb; q++) {
        const uint32_t* rx = rep_ptr(C, C.a + sB[q], 0, 0);
        const uint32_t* rz = rep_ptr(C, C.a + sB[q], 0, 1);
        x[0] ^= rx[0];
        z[0] ^= rz[0];
        if (C.W >= 2) {
            x[1] ^= rx[1];
            z[1] ^= rz[1];
        }
        const uint32_t fl = C.flags[C.a + sB[q]];
        P1 += fl & 1u;
        P2 += (fl >> 1) & 1u;
    }
}

DIST_HD bool use_fast(const LaneCtx& C, int i) {
    return DIST_FAST_PATH(i, C.proj);
}

// Combination ranks [lo, hi) that lane `lane` walks in warp-chunk `chunk`
// of segment sg (chunk_base <= chunk); false if the lane has none.
DIST_HD bool seg_lane_range(const SegDesc& sg, unsigned long long chunk, int lane, unsigned long long& lo,
                            unsigned long long& hi) {
    lo = sg.rank0 + ((chunk - sg.chunk_base) * 32ull + (unsigned long long)lane) * sg.spl;
    if (lo >= sg.rank1) return false;
    hi = lo + sg.spl < sg.rank1 ? lo + sg.spl : sg.rank1;
    return true;
}

// Walks the combination ranks [lo, hi) of segment sg; returns the number of
// codewords evaluated.  Sink provides peek() (current upper bound),
// record(...) and vote_any(p) (true if p holds on any lane running in step
// with this one).  u_first is a recent value of U the caller already holds,
// taken as the bound of the first subset, so that the lane does not wait for
// a fresh read before its first subset.  kTwo = false leaves out the two-word
// filter; a launch whose bound can never reach it (U - P <= t1 from the
// start) runs that instance, which needs fewer registers.  Either filter is
// a lower bound on the weight, so the instance changes no result.
template <class Sink, bool kTwo = true>
DIST_HD unsigned long long walk_range(const LaneCtx& C, Sink& sink, uint32_t& thr, const SegDesc& sg,
                                      unsigned long long lo, unsigned long long hi, uint32_t u_first,
                                      unsigned long long peek_mask = 0) {
    const int i = (int)sg.i, nb = (int)sg.r - i;
    uint8_t sA[DIST_MAXR], sB[DIST_MAXR], dig[DIST_MAXR];
    for (int p = 0; p < DIST_MAXR; p++) dig[p] = 0;
    // (no B-units in the subset: every rank is an A-rank, no 64-bit division)
    unsigned long long tB = sg.NB == 1 ? 0ull : lo / sg.NA, tA = lo - tB * sg.NA;
    rd_unrank(C.binom, C.bstride, C.b, tB, nb, sB);
    rd_unrank(C.binom, C.bstride, C.a, tA, i, sA);
    uint32_t vbx[2], vbz[2], PB1, PB2;
    b_words(C, nb, sB, vbx, vbz, PB1, PB2);
    const bool fast = use_fast(C, i);
    // per-segment and per-matrix constants of the subset loop, read once
    // (as references into shared memory they would be read every subset)
    const int L_before = sg.L_before, a = C.a;
    const unsigned long long codes = sg.codes, NA = sg.NA;
    const bool all_outside = (C.a_all & 1u) && (!kTwo || (C.a_all & 2u));
    unsigned long long done = 0;
    // The running bound is read one subset ahead: a stale (larger) value is
    // still a valid threshold, and the load's latency overlaps the work.
    // With peek_mask = 7 it is read only at every eighth subset: for a launch
    // whose bound already meets the estimate of d (it rarely falls further)
    // a read at every subset cost 4 % on the QC n = 72 launch (0.0722
    // against 0.0691 ms), while launches whose bound still falls need the
    // fresh value to stop early (small random codes solved one per launch
    // evaluated 35 % more codewords with the sparse reads).
    uint32_t u_next = u_first;
    for (unsigned long long idx = lo; idx < hi; ++idx) {
        const uint32_t u = u_next;
        if (((idx - lo) & peek_mask) == 0) u_next = sink.peek();
        thr = u < thr ? u : thr;
        if ((int)u <= L_before) break;
        if (fast) {
            // packages with a pivot outside the filtered words each add one
            // (P2 is read by the two-word filter only)
            uint32_t P1 = PB1, P2 = PB2;
            if (all_outside) {
                // every A-unit's pivot lies beyond the filtered words
                P1 += (uint32_t)i;
                P2 += (uint32_t)i;
            } else {
                for (int p = 0; p < i; p++) {
                    const uint32_t fl = C.flags[sA[p]];
                    P1 += fl & 1u;
                    P2 += (fl >> 1) & 1u;
                }
            }
            // two filter words while the bound is far above what word 0 can
            // rule out (decided together by the lanes running in step)
            const bool two = kTwo && sink.vote_any(C.W >= 2 && (int)thr - (int)P1 > C.t1);
            if (two) {
                if (P2 < thr) eval_fast<2>(C, sink, thr, i, sA, dig, nb, sB, vbx, vbz, P2);
            } else {
                if (P1 < thr) eval_fast<1>(C, sink, thr, i, sA, dig, nb, sB, vbx, vbz, P1);
            }
        } else {
            thr = eval_generic(C, sink, thr, i, sA, nb, sB);
        }
        done += codes;
        if (idx + 1 < hi) {
            if (++tA == NA) {
                tA = 0;
                rd_next(sB, nb, C.b);
                b_words(C, nb, sB, vbx, vbz, PB1, PB2);
                for (int p = 0; p < i; p++) sA[p] = (uint8_t)p;
            } else {
                rd_next(sA, i, a);
            }
        }
    }
    return done;
}

}  // namespace dist
