// iso.cpp -- host side of the isometry method (Algorithm 3): the image rows,
// the systematic matrices on disjoint information sets, the bound and the
// witness.
#include "iso.h"

#include <string.h>

#include <algorithm>

namespace dist {

namespace {

struct Row3 {
    uint32_t w[kIsoMaxWords];
};

inline int get3(const Row3& r, int i) { return (int)((r.w[i >> 5] >> (i & 31)) & 1u); }
inline void set3(Row3& r, int i) { r.w[i >> 5] |= 1u << (i & 31); }
inline void xor3(Row3& a, const Row3& b) {
    for (int t = 0; t < kIsoMaxWords; t++) a.w[t] ^= b.w[t];
}
inline void xorc(Coef& a, const Coef& b) {
    for (int q = 0; q < 2; q++)
        for (int t = 0; t < DIST_MAXCW; t++) a.p[q][t] ^= b.p[q][t];
}
inline int pbit(const uint32_t* v, int i) { return (int)((v[i >> 5] >> (i & 31)) & 1u); }

// iso(x, z) = (x, z, x + z), bit q of each block for qubit q.
Row3 image(const Vec& v, int n) {
    Row3 r;
    memset(&r, 0, sizeof r);
    for (int q = 0; q < n; q++) {
        const int x = pbit(v.x, q), z = pbit(v.z, q);
        if (x) set3(r, q);
        if (z) set3(r, n + q);
        if (x ^ z) set3(r, 2 * n + q);
    }
    return r;
}

bool outside(const Plan& p, const Coef& c) {
    if (p.n_stab == 0) return true;
    for (int w = 0; w < DIST_MAXCW; w++)
        if ((c.p[0][w] | c.p[1][w]) & p.outside[w]) return true;
    return false;
}

}  // namespace

int iso_build(const Plan& p, IsoPlan* ip) {
    *ip = IsoPlan();
    const int n = p.n, n3 = 3 * n;
    // F2 rows of the code with their coefficients over the basis: the basis
    // itself, or for an F4 basis row v both v (scalar 1) and alpha v (scalar
    // alpha), alpha (x, z) = (z, x + z).
    std::vector<Row3> base;
    std::vector<Coef> bcoef;
    for (int i = 0; i < p.k_eff; i++) {
        Coef c;
        memset(&c, 0, sizeof c);
        c.p[0][i >> 5] |= 1u << (i & 31);
        base.push_back(image(p.basis[i], n));
        bcoef.push_back(c);
        if (p.field == 4) {
            Vec a;
            memset(&a, 0, sizeof a);
            for (int w = 0; w < DIST_MAXW; w++) {
                a.x[w] = p.basis[i].z[w];
                a.z[w] = p.basis[i].x[w] ^ p.basis[i].z[w];
            }
            Coef ca;
            memset(&ca, 0, sizeof ca);
            ca.p[1][i >> 5] |= 1u << (i & 31);
            base.push_back(image(a, n));
            bcoef.push_back(ca);
        }
    }
    const int K = (int)base.size();
    if (K == 0) return P_EZERO;
    if (K > DIST_MAXK) return P_ERANGE;
    ip->K = K;
    ip->n3 = n3;
    std::vector<char> used(n3, 0);
    ip->u0 = DIST_WINF;
    while ((int)ip->G.size() < DIST_MAXGAMMA) {
        // reduced echelon form of the basis on the columns still unused
        std::vector<Row3> R = base;
        std::vector<Coef> C = bcoef;
        std::vector<int> pivcol;
        int row = 0;
        for (int col = 0; col < n3 && row < K; col++) {
            if (used[col]) continue;
            int q = -1;
            for (int i = row; i < K; i++)
                if (get3(R[i], col)) {
                    q = i;
                    break;
                }
            if (q < 0) continue;
            std::swap(R[q], R[row]);
            std::swap(C[q], C[row]);
            for (int i = 0; i < K; i++)
                if (i != row && get3(R[i], col)) {
                    xor3(R[i], R[row]);
                    xorc(C[i], C[row]);
                }
            pivcol.push_back(col);
            row++;
        }
        if (row == 0) break;
        IsoGamma g;
        g.k = row;
        g.f = K - row;
        std::vector<char> isp(n3, 0);
        for (int c : pivcol) isp[c] = 1;
        std::vector<int> rest;  // columns outside this matrix's information set
        for (int c = 0; c < n3; c++)
            if (!isp[c]) rest.push_back(c);
        g.words = std::max(1, ((int)rest.size() + 31) / 32);
        g.rows.assign((size_t)K * g.words, 0);
        g.piv.assign(K, 0);
        g.coef = C;
        for (int i = 0; i < K; i++) {
            g.piv[i] = i < row ? 1 : 0;
            uint32_t* dst = &g.rows[(size_t)i * g.words];
            for (size_t t = 0; t < rest.size(); t++)
                if (get3(R[i], rest[t])) dst[t >> 5] |= 1u << (t & 31);
            int w = g.piv[i];
            for (int t = 0; t < g.words; t++) w += __builtin_popcount(dst[t]);
            if (w < ip->u0 && outside(p, C[i])) {
                ip->u0 = w;
                ip->u0_g = (int)ip->G.size();
                ip->u0_row = i;
            }
        }
        for (int c : pivcol) used[c] = 1;
        ip->words = std::max(ip->words, g.words);
        ip->G.push_back(std::move(g));
    }
    return ip->G.empty() ? P_EZERO : P_OK;
}

int iso_lower_bound(const IsoPlan& ip, int r, int jpos) {
    long L = 0;
    for (size_t t = 0; t < ip.G.size(); t++) {
        const int rr = (int)t <= jpos ? r : r - 1;
        if (rr >= ip.K) return DIST_WINF;  // every combination of its rows seen
        L += std::max(0, rr + 1 - ip.G[t].f);
    }
    return (int)std::min<long>(L, DIST_WINF - 1);
}

int iso_decode(const Plan& p, const IsoPlan& ip, int g, const uint8_t* rows, int count, int wH,
               uint8_t* witness, uint8_t* coeffs) {
    if (g < 0 || g >= (int)ip.G.size() || count < 1 || (wH & 1)) return P_EINVAL;
    const IsoGamma& G = ip.G[g];
    Coef k;
    memset(&k, 0, sizeof k);
    int w = 0;
    std::vector<uint32_t> acc(G.words, 0);
    for (int t = 0; t < count; t++) {
        if (rows[t] >= ip.K) return P_EINVAL;
        xorc(k, G.coef[rows[t]]);
        w += G.piv[rows[t]];
        for (int q = 0; q < G.words; q++) acc[q] ^= G.rows[(size_t)rows[t] * G.words + q];
    }
    for (int q = 0; q < G.words; q++) w += __builtin_popcount(acc[q]);
    if (w != wH) return P_EINVAL;
    // wt_H of the image is twice the symplectic weight of the codeword
    return plan_decode_coef(p, k, wH / 2, witness, coeffs);
}

}  // namespace dist
