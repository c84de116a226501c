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
// Order of representatives (the fast path): the three largest units of the
// subset form a 27-entry table of word-0 partial sums held in registers; the
// other units' digits advance by a modular ternary Gray code (step k changes
// digit nu_3(k) by +1 mod 3, which XORs the unit's third representative,
// since rep0 ^ rep1 ^ rep2 = 0).  Every codeword then costs two LOP3, one
// POPC and one min on word 0 of each plane.  Word 0 holds the qubits that are
// not pivots of this matrix, so popc(word 0) is a sharp lower bound on the
// weight; only when it falls below the current upper bound is the full
// weight computed (the slow path), which keeps the result exact.
#pragma once
#include "dist_types.h"

namespace dist {

#if defined(__CUDACC__)
#define DIST_HD_COLD __host__ __device__ __noinline__
#define DIST_HD_HOT __host__ __device__ __noinline__
#else
#define DIST_HD_COLD inline
#define DIST_HD_HOT inline
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

DIST_HD unsigned long long binom_at(const unsigned long long* B, int n, int k) {
    if (k < 0 || n < k) return 0ull;
    return B[n * (DIST_MAXR + 1) + k];
}

// Subset of revolving-door rank R, t elements, written ascending into s.
DIST_HD void rd_unrank(const unsigned long long* B, unsigned long long R, int t, uint8_t* s) {
    for (int tt = t; tt >= 1; --tt) {
        int lo = tt - 1, hi = DIST_MAXU;  // C(lo, tt) <= R < C(hi, tt)
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (binom_at(B, mid, tt) <= R) lo = mid;
            else hi = mid;
        }
        s[tt - 1] = (uint8_t)lo;
        R = binom_at(B, lo + 1, tt) - 1 - R;
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

// What a lane reads.  reps / r0 live in shared memory on the device.
struct LaneCtx {
    const uint32_t* reps;              // [u][3][2][W]
    const U2* r0;                      // [a][3]: word 0 of the A-units' representatives
    const uint32_t* coefs;             // [u][3][2][CW]
    const unsigned long long* binom;
    const uint32_t* outside;
    int a, b, W, CW, r, gamma, proj, exclude;
};

DIST_HD const uint32_t* rep_ptr(const LaneCtx& C, int unit, int e, int plane) {
    return C.reps + ((unit * 3 + e) * 2 + plane) * C.W;
}

// Exact weight of the combination (A-units sA with digits eA, B-units sB);
// records it when it beats thr and, in exclusion mode, lies outside S.
template <class Sink>
DIST_HD_COLD void consider(const LaneCtx& C, Sink& sink, uint32_t& thr, int i, const uint8_t* sA,
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
    if (wt >= thr) return;
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
        if (!acc) return;  // inside S = span(first n_stab rows)
    }
    thr = wt;
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
}

// Every representative choice of one subset, each weighed exactly (small i).
template <class Sink>
DIST_HD_COLD void eval_generic(const LaneCtx& C, Sink& sink, uint32_t& thr, int i, const uint8_t* sA,
                          int nb, const uint8_t* sB) {
    uint8_t e[DIST_MAXR];
    for (int p = 0; p < i; p++) e[p] = 0;
    const int first = C.proj ? 1 : 0;
    for (;;) {
        consider(C, sink, thr, i, sA, e, nb, sB);
        int p = first;
        while (p < i && e[p] == 2) {
            e[p] = 0;
            ++p;
        }
        if (p >= i) break;
        ++e[p];
    }
}

// Slow path of one 27-codeword block: every entry whose word-0 weight is
// below thr is weighed in full.
template <class Sink>
DIST_HD_COLD void block_slow(const LaneCtx& C, Sink& sink, uint32_t& thr, int i, const uint8_t* sA,
                        const uint8_t* dig, int nb, const uint8_t* sB, uint32_t bx, uint32_t bz) {
    const int p0 = i - 3;
    uint8_t e[DIST_MAXR];
    for (int p = 0; p < p0; p++) e[p] = dig[p];
    for (int j = 0; j < 27; j++) {
        const int e0 = j % 3, e1 = (j / 3) % 3, e2 = j / 9;
        const U2 ta = C.r0[sA[p0] * 3 + e0], tb = C.r0[sA[p0 + 1] * 3 + e1],
                 tc = C.r0[sA[p0 + 2] * 3 + e2];
        uint32_t t = (bx ^ ta.x ^ tb.x ^ tc.x) | (bz ^ ta.z ^ tb.z ^ tc.z);
        if ((uint32_t)popc32(t) >= thr) continue;
        e[p0] = (uint8_t)e0;
        e[p0 + 1] = (uint8_t)e1;
        e[p0 + 2] = (uint8_t)e2;
        consider(C, sink, thr, i, sA, e, nb, sB);
    }
}

// Fast path: subsets with at least three varying units.  Kept out of line so
// that only its own state (the table, the base word and the counters) is live
// in the inner loop.
template <class Sink>
DIST_HD_HOT void eval_fast(const LaneCtx& C, Sink& sink, uint32_t& thr, int i, const uint8_t* sA,
                       uint8_t* dig, int nb, const uint8_t* sB, uint32_t vbx, uint32_t vbz) {
    const int p0 = i - 3;
    uint32_t Tx[27], Tz[27];
    {
        const U2* ra = C.r0 + sA[p0] * 3;
        const U2* rb = C.r0 + sA[p0 + 1] * 3;
        const U2* rc = C.r0 + sA[p0 + 2] * 3;
        U2 A[3], B[3], Cc[3];
#pragma unroll
        for (int e = 0; e < 3; e++) {
            A[e] = ra[e];
            B[e] = rb[e];
            Cc[e] = rc[e];
        }
#pragma unroll
        for (int e2 = 0; e2 < 3; e2++)
#pragma unroll
            for (int e1 = 0; e1 < 3; e1++)
#pragma unroll
                for (int e0 = 0; e0 < 3; e0++) {
                    Tx[e2 * 9 + e1 * 3 + e0] = Cc[e2].x ^ B[e1].x ^ A[e0].x;
                    Tz[e2 * 9 + e1 * 3 + e0] = Cc[e2].z ^ B[e1].z ^ A[e0].z;
                }
    }
    uint32_t bx = vbx, bz = vbz;
    for (int p = 0; p < p0; p++) {
        const U2 v = C.r0[sA[p] * 3 + dig[p]];
        bx ^= v.x;
        bz ^= v.z;
    }
    const int first = C.proj ? 1 : 0;
    const int nouter = p0 - first;
    uint32_t nk = 1;
    for (int q = 0; q < nouter; q++) nk *= 3u;
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
            const U2 v = C.r0[sA[p] * 3 + (e == 0 ? 2 : e - 1)];
            bx ^= v.x;
            bz ^= v.z;
            dig[p] = (uint8_t)(e == 2 ? 0 : e + 1);
        }
        uint32_t m0 = 0xFFFFu, m1 = 0xFFFFu;
#pragma unroll
        for (int j = 0; j < 27; j++) {
            const uint32_t t = (bx ^ Tx[j]) | (bz ^ Tz[j]);
            const uint32_t c = (uint32_t)popc32(t);
            if (j & 1) m1 = c < m1 ? c : m1;
            else m0 = c < m0 ? c : m0;
        }
        const uint32_t m = m0 < m1 ? m0 : m1;
        if (m < thr) block_slow(C, sink, thr, i, sA, dig, nb, sB, bx, bz);
    }
}

// Word 0 of the sum of the chosen B-units' single representatives.
DIST_HD void b_word0(const LaneCtx& C, int nb, const uint8_t* sB, uint32_t& x, uint32_t& z) {
    x = z = 0;
    for (int q = 0; q < nb; q++) {
        x ^= rep_ptr(C, C.a + sB[q], 0, 0)[0];
        z ^= rep_ptr(C, C.a + sB[q], 0, 1)[0];
    }
}

DIST_HD bool use_fast(const LaneCtx& C, int i) {
    return i >= 3 + C.proj && i - 3 - C.proj <= DIST_FAST_MAX_OUTER;
}

// Walks the combination ranks [lo, hi) of segment sg; returns the number of
// codewords evaluated.  Sink provides poll(thr) -> stop? and record(...).
template <class Sink>
DIST_HD unsigned long long walk_range(const LaneCtx& C, Sink& sink, uint32_t& thr, const SegDesc& sg,
                                      unsigned long long lo, unsigned long long hi) {
    const int i = (int)sg.i, nb = C.r - i;
    uint8_t sA[DIST_MAXR], sB[DIST_MAXR], dig[DIST_MAXR];
    for (int p = 0; p < DIST_MAXR; p++) dig[p] = 0;
    unsigned long long tB = lo / sg.NA, tA = lo - tB * sg.NA;
    rd_unrank(C.binom, tB, nb, sB);
    rd_unrank(C.binom, tA, i, sA);
    uint32_t vbx, vbz;
    b_word0(C, nb, sB, vbx, vbz);
    const bool fast = use_fast(C, i);
    unsigned long long done = 0;
    for (unsigned long long idx = lo; idx < hi; ++idx) {
        if (sink.poll(thr)) break;
        if (fast) eval_fast(C, sink, thr, i, sA, dig, nb, sB, vbx, vbz);
        else eval_generic(C, sink, thr, i, sA, nb, sB);
        done += sg.codes;
        if (idx + 1 < hi) {
            if (++tA == sg.NA) {
                tA = 0;
                rd_next(sB, nb, C.b);
                b_word0(C, nb, sB, vbx, vbz);
                for (int p = 0; p < i; p++) sA[p] = (uint8_t)p;
            } else {
                rd_next(sA, i, C.a);
            }
        }
    }
    return done;
}

}  // namespace dist
