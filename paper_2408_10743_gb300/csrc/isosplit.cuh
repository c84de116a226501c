// isosplit.cuh -- the split walk of the isometry kernel (host and device).
//
// Round r of a systematic matrix visits the sum of every r-subset of its K
// rows.  Cut the rows into two halves, H0 = rows [0, K0) and H1 = rows
// [K0, K).  An r-subset meets H0 in some i rows and H1 in the other r - i,
// and those two parts determine it, so round r is the disjoint union over i
// of the products
//     { sum(S0) + sum(S1) : S0 an i-subset of H0, S1 an (r - i)-subset of H1 },
// one *term* per i.  In a term, the side with fewer subsets is the tile side:
// a block stages the sums of a range of its subsets in shared memory.  The
// other is the lane side: each thread holds the sums of kSplitNB consecutive
// subsets in registers, stepping from one to the next in colexicographic
// order.  Every pair (tile entry, register value) is one codeword, so a
// codeword costs two XORs, two popcounts and an add, and one broadcast table
// read serves kSplitNB codewords.
//
// A term is cut into units: a range of tile-side subsets (tile_span) times a
// range of lane-side subsets (kSplitThreads x kSplitNB x groups).  A term
// whose tile side is short (at most kSplitTile subsets) takes all of it in
// one unit and gives each thread `groups` register sets one after another;
// the others take one register set per thread and a tile range staged
// kSplitTile entries at a time.  Blocks claim units in order, the terms with
// the longest tile side first.
//
// Host and device: the kernel (iso.cu) and the test harness that checks on
// the CPU that the units cover every r-subset exactly once use these same
// functions.
#pragma once
#include <string.h>

#include "dist_types.h"
#include "packed.cuh"

namespace dist {

constexpr int kSplitThreads = 256;  // threads of a block
constexpr int kSplitNB = 8;         // register values of a thread
constexpr int kSplitTile = 256;     // tile entries staged at a time
constexpr int kSplitMaxT = 8;       // rows of one side (packed in 64 bits)
constexpr int kSplitMaxTerms = 3 * kSplitMaxT + 1;  // a split, and one more of its two one-sided terms

// Words 0-2 of a sum of rows (on the columns outside the information set)
// and its pivot count; as a neighbour delta, rows c and c + 1 XORed and the
// change of the pivot count (modulo 2^32).
struct alignas(16) SplitRow {
    uint32_t x, y, z, np;
};

DIST_HD void split_add(SplitRow* a, const SplitRow& b) {
    a->x ^= b.x;
    a->y ^= b.y;
    a->z ^= b.z;
    a->np += b.np;
}

struct SplitTerm {
    unsigned long long n_tile, n_lane;  // subsets of each side
    unsigned long long unit0, units;    // first unit of the term, units
    uint32_t nh;                        // tile ranges: ceil(n_tile / tile_span)
    uint32_t tile_span;                 // tile-side subsets per unit
    uint32_t groups;                    // register sets per thread per unit
    uint8_t tile_off, tile_kh, tile_t;  // tile side: first row, rows of its half, subset size
    uint8_t lane_off, lane_kh, lane_t;  // lane side
    uint8_t pad[2];
};

struct SplitPlan {
    SplitTerm term[kSplitMaxTerms];
    int nterms = 0;
    unsigned long long units = 0;
};

// Unit u of a launch: its term, its tile-side range [t_lo, t_hi), its
// lane-side range [l_lo, l_hi) and the lane-side subsets per thread (`per`:
// thread j takes [l_lo + j per, l_lo + (j + 1) per) within the range).
struct SplitUnit {
    int term;
    unsigned long long t_lo, t_hi, l_lo, l_hi, per;
};

DIST_HD SplitUnit split_unit(const SplitTerm* terms, int nterms, unsigned long long u) {
    SplitUnit U;
    int e = 0;
    while (e + 1 < nterms && u >= terms[e + 1].unit0) ++e;
    const SplitTerm& S = terms[e];
    const unsigned long long ul = u - S.unit0;
    const unsigned long long h = ul % S.nh, g = ul / S.nh;
    U.term = e;
    U.t_lo = h * S.tile_span;
    U.t_hi = U.t_lo + S.tile_span < S.n_tile ? U.t_lo + S.tile_span : S.n_tile;
    U.per = (unsigned long long)kSplitNB * S.groups;
    U.l_lo = g * U.per * kSplitThreads;
    U.l_hi = U.l_lo + U.per * kSplitThreads < S.n_lane ? U.l_lo + U.per * kSplitThreads : S.n_lane;
    return U;
}

// Largest c in [lo, hi] with C(c, t) <= R, by bisection (C(hi + 1, t) taken
// as infinite).  B is the binomial table, row c, column t.
DIST_HD int split_top(const unsigned long long* B, int t, unsigned long long R, int lo, int hi) {
    int a = lo, b = hi + 1;
    while (b - a > 1) {
        const int mid = (a + b) >> 1;
        if (B[mid * (DIST_MAXR + 1) + t] <= R) a = mid;
        else b = mid;
    }
    return a;
}

// The t-subset of colexicographic rank R of the half [off, off + kh): its
// elements (local indices, ascending, packed) and the sum of its rows.
DIST_HD void split_unrank(const unsigned long long* B, const SplitRow* rows, int off, int kh, int t,
                          unsigned long long R, uint64_t* T, SplitRow* sum) {
    uint64_t S = 0;
    SplitRow v = {0u, 0u, 0u, 0u};
    int hi = kh - 1;
    for (int e = t; e >= 1; --e) {
        const int c = split_top(B, e, R, e - 1, hi);
        S = pk_put(S, e - 1, c);
        R -= B[c * (DIST_MAXR + 1) + e];
        split_add(&v, rows[off + c]);
        hi = c - 1;
    }
    *T = S;
    *sum = v;
}

// The same subset as row indices (off + local), for a witness.
DIST_HD void split_rows(const unsigned long long* B, int off, int kh, int t, unsigned long long R, uint8_t* s) {
    int hi = kh - 1;
    for (int e = t; e >= 1; --e) {
        const int c = split_top(B, e, R, e - 1, hi);
        s[e - 1] = (uint8_t)(off + c);
        R -= B[c * (DIST_MAXR + 1) + e];
        hi = c - 1;
    }
}

// Colexicographic successor of the t-subset T of the half starting at row
// off, with its sum: the lowest element that can move up by one does, and
// the ones below it return to 0, 1, ...  The caller never steps past the
// last subset.  `delta` holds rows c and c + 1 XORed (the row after the
// half's last is never used: an element moves up only below the next one or
// below the half's end).
DIST_HD void split_next(const SplitRow* rows, const SplitRow* delta, int off, int t, uint64_t* T, SplitRow* sum) {
    uint64_t S = *T;
    SplitRow v = *sum;
    int e = 0;
    while (e + 1 < t && pk_get(S, e) + 1 == pk_get(S, e + 1)) ++e;
    for (int u = 0; u < e; ++u) {  // elements below e form a run ending at s_e - 1; they restart at u
        const SplitRow qo = rows[off + pk_get(S, u)], qn = rows[off + u];
        v.x ^= qo.x ^ qn.x;
        v.y ^= qo.y ^ qn.y;
        v.z ^= qo.z ^ qn.z;
        v.np += qn.np - qo.np;
        S = pk_put(S, u, u);
    }
    const int c = pk_get(S, e);
    split_add(&v, delta[off + c]);
    S = pk_put(S, e, c + 1);
    *T = S;
    *sum = v;
}

// Plans round r of a K-row matrix as split terms, each cut into units of
// about `target` codewords' worth of work.  B is the binomial table (host
// copy).  Returns false if the split walk does not apply (r outside
// [1, kSplitMaxT], K < 2 or K > 256).
//
// The terms i = 0 and i = r of a split have a tile side of one subset (the
// empty one): every register value would meet a single tile entry.  Such a
// term is all t-subsets of one half, so it is split again in the same way
// (once: kSplitDepth) when it holds at least kSplitResplit codewords; its own
// one-sided terms are kept.  Units of a term with a short tile side hold
// fewer codewords, in proportion to the extra cost of stepping its register
// values (about kSplitStepCost tile entries' worth per value).
constexpr int kSplitDepth = 1;
constexpr unsigned long long kSplitResplit = 1ull << 16;
constexpr int kSplitStepCost = 4;

inline bool split_plan(int K, int r, unsigned long long target, const unsigned long long* B, SplitPlan* sp) {
    sp->nterms = 0;
    sp->units = 0;
    if (r < 1 || r > kSplitMaxT || K < 2 || K > 256) return false;
    auto binom = [&](int n, int k) -> unsigned long long {
        return k < 0 || k > n ? 0ull : B[n * (DIST_MAXR + 1) + k];
    };
    const unsigned long long lane1 = (unsigned long long)kSplitThreads * kSplitNB;
    int n = 0;
    auto add = [&](int off0, int k0, int t0, int off1, int k1, int t1) {
        const unsigned long long n0 = binom(k0, t0), n1 = binom(k1, t1);
        SplitTerm& S = sp->term[n++];
        memset(&S, 0, sizeof S);
        const bool tile0 = n0 <= n1;  // the side with fewer subsets is staged
        S.n_tile = tile0 ? n0 : n1;
        S.n_lane = tile0 ? n1 : n0;
        S.tile_off = (uint8_t)(tile0 ? off0 : off1);
        S.tile_kh = (uint8_t)(tile0 ? k0 : k1);
        S.tile_t = (uint8_t)(tile0 ? t0 : t1);
        S.lane_off = (uint8_t)(tile0 ? off1 : off0);
        S.lane_kh = (uint8_t)(tile0 ? k1 : k0);
        S.lane_t = (uint8_t)(tile0 ? t1 : t0);
        if (S.n_tile <= (unsigned long long)kSplitTile) {
            S.tile_span = (uint32_t)S.n_tile;
            const unsigned long long cw = (S.n_tile + kSplitStepCost) * lane1;  // work of one register set per thread
            const unsigned long long g = (target + cw - 1) / cw;
            const unsigned long long gmax = (S.n_lane + lane1 - 1) / lane1;
            S.groups = (uint32_t)(g < 1 ? 1 : g > gmax ? gmax : g);
        } else {
            unsigned long long span = (target + lane1 - 1) / lane1;
            span = (span + 63) / 64 * 64;
            if (span < 64) span = 64;
            if (span > S.n_tile) span = S.n_tile;
            if (span > (1ull << 20)) span = 1ull << 20;
            S.tile_span = (uint32_t)span;
            S.groups = 1;
        }
        S.nh = (uint32_t)((S.n_tile + S.tile_span - 1) / S.tile_span);
        const unsigned long long lane_span = lane1 * S.groups;
        S.units = (unsigned long long)S.nh * ((S.n_lane + lane_span - 1) / lane_span);
    };
    // ranges (off, kh, t, depth): all t-subsets of rows [off, off + kh)
    int stk[2 * kSplitDepth + 2][4];
    int ns = 0;
    stk[ns][0] = 0, stk[ns][1] = K, stk[ns][2] = r, stk[ns][3] = 0, ns++;
    while (ns > 0) {
        --ns;
        const int off = stk[ns][0], kh = stk[ns][1], t = stk[ns][2], depth = stk[ns][3];
        const int k0 = kh / 2, k1 = kh - k0;
        for (int i = 0; i <= t; i++) {
            if (binom(k0, i) == 0 || binom(k1, t - i) == 0) continue;
            const bool one_sided = i == 0 || i == t;
            const int roff = i == 0 ? off + k0 : off, rk = i == 0 ? k1 : k0;
            if (one_sided && t >= 2 && depth < kSplitDepth && rk >= 2 && binom(rk, t) >= kSplitResplit) {
                stk[ns][0] = roff, stk[ns][1] = rk, stk[ns][2] = t, stk[ns][3] = depth + 1, ns++;
                continue;
            }
            add(off, k0, i, off + k0, k1, t - i);
        }
    }
    // longest tile side first: the terms with short tile sides, whose units
    // are sized by `groups`, come last and fill the end of the launch
    for (int a = 1; a < n; a++)
        for (int b = a; b > 0 && sp->term[b].n_tile > sp->term[b - 1].n_tile; b--) {
            const SplitTerm tmp = sp->term[b];
            sp->term[b] = sp->term[b - 1];
            sp->term[b - 1] = tmp;
        }
    unsigned long long u0 = 0;
    for (int a = 0; a < n; a++) {
        sp->term[a].unit0 = u0;
        u0 += sp->term[a].units;
    }
    sp->nterms = n;
    sp->units = u0;
    return true;
}

}  // namespace dist
