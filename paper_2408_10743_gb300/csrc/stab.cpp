// stab.cpp -- front end for qubit stabilizer codes (host only, no CUDA).
//
// A stabilizer code Q = [[n, k, d(Q)]] is given by generators of its
// classical stabilizer code S in F2^{2n}, with S inside its symplectic dual.
// The dual N = S^{perp_s} (the classical normalizer code, of dimension
// n + k) is what the distance search enumerates (Section 2): d(Q) is the
// least symplectic weight on N minus S when k > 0, and on S itself when
// k = 0.  This file builds a generator matrix of N whose first rows are a
// basis of S -- the row order the exclusion check of the modified
// Brouwer-Zimmermann algorithm (Section 2.1) expects.
#include <stdint.h>
#include <string.h>

#include <vector>

#include "plan.h"

namespace dist {

namespace {

constexpr int kWords = (2 * DIST_MAXN + 63) / 64;  // a row of 2n bits

struct Row {
    uint64_t w[kWords];
};

inline int get(const Row& r, int i) { return (int)((r.w[i >> 6] >> (i & 63)) & 1u); }
inline void put(Row& r, int i) { r.w[i >> 6] |= 1ull << (i & 63); }
inline void add(Row& a, const Row& b) {
    for (int t = 0; t < kWords; t++) a.w[t] ^= b.w[t];
}
inline bool zero(const Row& a) {
    for (int t = 0; t < kWords; t++)
        if (a.w[t]) return false;
    return true;
}

// Symplectic form (a, b) . (c, d) = a.d + b.c over F2; bit i < n is x_i,
// bit n + i is z_i.
int symp(const Row& u, const Row& v, int n) {
    int s = 0;
    for (int i = 0; i < n; i++) s ^= (get(u, i) & get(v, n + i)) ^ (get(u, n + i) & get(v, i));
    return s;
}

// Incremental echelon basis: insert(v) reduces v against the basis and keeps
// it if it is independent.
struct Echelon {
    std::vector<Row> rows;
    std::vector<int> piv;
    bool insert(Row v, int nbits) {
        for (size_t e = 0; e < rows.size(); e++)
            if (get(v, piv[e])) add(v, rows[e]);
        if (zero(v)) return false;
        int q = 0;
        while (q < nbits && !get(v, q)) q++;
        // keep the basis reduced at the new pivot
        for (size_t e = 0; e < rows.size(); e++)
            if (get(rows[e], q)) add(rows[e], v);
        rows.push_back(v);
        piv.push_back(q);
        return true;
    }
};

}  // namespace

int stab_normalizer(const uint8_t* stab, int n, int m, std::vector<uint8_t>* gen, int* K_out,
                    int* n_stab_out) {
    if (!stab || !gen || n < 1 || n > DIST_MAXN || m < 1) return P_EINVAL;
    const int nb = 2 * n;
    // S1: the given generators, reduced to a basis of S (in input order)
    std::vector<Row> S;
    Echelon span_s;
    for (int r = 0; r < m; r++) {
        Row v;
        memset(&v, 0, sizeof v);
        for (int i = 0; i < nb; i++) {
            const uint8_t b = stab[(size_t)r * nb + i];
            if (b > 1) return P_EINVAL;
            if (b) put(v, i);
        }
        if (span_s.insert(v, nb)) S.push_back(v);
    }
    const int s = (int)S.size();
    if (s == 0) return P_EZERO;
    // S must lie in its symplectic dual (the generators commute)
    for (int i = 0; i < s; i++)
        for (int j = i + 1; j < s; j++)
            if (symp(S[i], S[j], n)) return P_EINVAL;
    std::vector<Row> out = S;
    int n_stab = s;
    if (s < n) {
        // N = { v : symp(b, v) = 0 for every basis row b of S }: the null space
        // of the rows (b_z | b_x), from their reduced echelon form
        Echelon M;
        for (const Row& b : S) {
            Row t;
            memset(&t, 0, sizeof t);
            for (int i = 0; i < n; i++) {
                if (get(b, n + i)) put(t, i);
                if (get(b, i)) put(t, n + i);
            }
            M.insert(t, nb);
        }
        std::vector<char> is_piv(nb, 0);
        for (int q : M.piv) is_piv[q] = 1;
        // one null-space vector per free column f: bit f, plus bit piv[e] for
        // every echelon row e with a 1 at f
        Echelon span_n = span_s;
        for (int f = 0; f < nb; f++) {
            if (is_piv[f]) continue;
            Row v;
            memset(&v, 0, sizeof v);
            put(v, f);
            for (size_t e = 0; e < M.rows.size(); e++)
                if (get(M.rows[e], f)) put(v, M.piv[e]);
            // logical operators: null-space vectors outside the span so far
            if (span_n.insert(v, nb)) out.push_back(v);
        }
        if ((int)out.size() != nb - s) return P_EINVAL;  // cannot happen for commuting S
    } else {
        n_stab = 0;  // k = 0: d(Q) is the minimum weight of S itself
    }
    const int K = (int)out.size();
    gen->assign((size_t)K * nb, 0);
    for (int r = 0; r < K; r++)
        for (int i = 0; i < nb; i++) (*gen)[(size_t)r * nb + i] = (uint8_t)get(out[r], i);
    *K_out = K;
    *n_stab_out = n_stab;
    return P_OK;
}

}  // namespace dist
