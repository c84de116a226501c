// plan.cpp -- host planner: ingest, package diagonalization, bound schedule,
// work description per launch, witness decoding.  Plain C++, no CUDA.
#include "plan.h"

#include <math.h>
#include <string.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>

namespace dist {

static std::atomic<int> g_chunks_per_warp{6}, g_lane_cap_log2{14}, g_lane_floor_log2{12};

Tuning tuning_get() {
    Tuning t;
    t.chunks_per_warp = g_chunks_per_warp.load();
    t.lane_cap_log2 = g_lane_cap_log2.load();
    t.lane_floor_log2 = g_lane_floor_log2.load();
    return t;
}

void tuning_set(const Tuning& t) {
    g_chunks_per_warp.store(std::max(1, std::min(t.chunks_per_warp, 256)));
    const int cap = std::max(8, std::min(t.lane_cap_log2, 24));
    g_lane_cap_log2.store(cap);
    g_lane_floor_log2.store(std::max(1, std::min(t.lane_floor_log2, cap)));
}

// ---------------------------------------------------------------------------
// Bit-plane helpers.
// ---------------------------------------------------------------------------
static inline int bit(const uint32_t* v, int i) { return (int)((v[i >> 5] >> (i & 31)) & 1u); }
static inline void setb(uint32_t* v, int i) { v[i >> 5] |= 1u << (i & 31); }

static inline void vxor(Vec& a, const Vec& b) {
    for (int w = 0; w < DIST_MAXW; w++) {
        a.x[w] ^= b.x[w];
        a.z[w] ^= b.z[w];
    }
}
static inline void cxor(Coef& a, const Coef& b) {
    for (int q = 0; q < 2; q++)
        for (int w = 0; w < DIST_MAXCW; w++) a.p[q][w] ^= b.p[q][w];
}
static inline bool vzero(const Vec& a) {
    for (int w = 0; w < DIST_MAXW; w++)
        if (a.x[w] | a.z[w]) return false;
    return true;
}

int vec_weight(const Vec& v, int W) {
    int s = 0;
    for (int w = 0; w < W; w++) s += __builtin_popcount(v.x[w] | v.z[w]);
    return s;
}

// Value of coordinate q as 0..3 = x_q + 2 z_q: the projection of a row onto
// qubit q (F2^2), or its F4 symbol.
static inline int proj(const Vec& v, int q) { return bit(v.x, q) | (bit(v.z, q) << 1); }

// F4 scalar c (1 = 1, 2 = alpha, 3 = alpha^2) times a plane pair (x, z) that
// encodes x + alpha z:  alpha (x + alpha z) = z + alpha (x + z).
static inline void f4_scale_planes(uint32_t* x, uint32_t* z, int nw, int c) {
    for (int w = 0; w < nw; w++) {
        uint32_t a = x[w], b = z[w];
        if (c == 2) {
            x[w] = b;
            z[w] = a ^ b;
        } else if (c == 3) {
            x[w] = a ^ b;
            z[w] = a;
        }
    }
}
static inline Vec vscale(const Vec& v, int c) {
    Vec r = v;
    f4_scale_planes(r.x, r.z, DIST_MAXW, c);
    return r;
}
static inline Coef cscale(const Coef& v, int c) {
    Coef r = v;
    f4_scale_planes(r.p[0], r.p[1], DIST_MAXCW, c);
    return r;
}
static inline int f4_inv(int c) { return c == 1 ? 1 : (c == 2 ? 3 : 2); }

// ---------------------------------------------------------------------------
// Binomials.
// ---------------------------------------------------------------------------
void binom_table(unsigned long long* tab) {
    const unsigned long long SAT = ~0ull;
    for (int n = 0; n <= DIST_MAXU; n++)
        for (int k = 0; k <= DIST_MAXR; k++) {
            unsigned long long v;
            if (k == 0) v = 1;
            else if (n == 0) v = 0;
            else {
                unsigned long long a = tab[(n - 1) * (DIST_MAXR + 1) + k - 1];
                unsigned long long b = tab[(n - 1) * (DIST_MAXR + 1) + k];
                v = (a == SAT || b == SAT || a + b < a) ? SAT : a + b;
            }
            tab[n * (DIST_MAXR + 1) + k] = v;
        }
}

static double dbinom(int n, int k) {
    if (k < 0 || k > n) return 0.0;
    return exp(lgamma(n + 1.0) - lgamma(k + 1.0) - lgamma(n - k + 1.0));
}

// C(n, k) exactly, or ~0 if it exceeds 2^63.  n <= DIST_MAXU and
// k <= DIST_MAXR (every launch's sizes) come from a table built once by the
// recurrence C(n, k) = C(n-1, k-1) + C(n-1, k), which saturates the same way.
static unsigned long long ubinom_loop(int n, int k) {
    if (k < 0 || k > n) return 0;
    if (k > n - k) k = n - k;
    unsigned __int128 v = 1;
    for (int i = 1; i <= k; i++) {
        v = v * (unsigned)(n - k + i) / (unsigned)i;
        if (v > ((unsigned __int128)1 << 63)) return ~0ull;
    }
    return (unsigned long long)v;
}

static unsigned long long ubinom(int n, int k) {
    if (k < 0 || k > n) return 0;
    if (n > DIST_MAXU || k > DIST_MAXR) return ubinom_loop(n, k);
    static const std::vector<unsigned long long> tab = [] {
        const unsigned long long SAT = ~0ull, LIM = 1ull << 63;
        std::vector<unsigned long long> t((size_t)(DIST_MAXU + 1) * (DIST_MAXR + 1), 0);
        for (int m = 0; m <= DIST_MAXU; m++)
            for (int j = 0; j <= DIST_MAXR && j <= m; j++) {
                unsigned long long v = 1;
                if (j > 0 && j < m) {
                    const unsigned long long a = t[(size_t)(m - 1) * (DIST_MAXR + 1) + j - 1];
                    const unsigned long long b = t[(size_t)(m - 1) * (DIST_MAXR + 1) + j];
                    const unsigned __int128 sum = (unsigned __int128)a + b;
                    v = (a == SAT || b == SAT || sum > LIM) ? SAT : (unsigned long long)sum;
                }
                t[(size_t)m * (DIST_MAXR + 1) + j] = v;
            }
        return t;
    }();
    return tab[(size_t)n * (DIST_MAXR + 1) + k];
}

static unsigned long long upow3(int e) {
    unsigned long long v = 1;
    for (int i = 0; i < e; i++) {
        if (v > (1ull << 62) / 3) return ~0ull;
        v *= 3;
    }
    return v;
}

// ---------------------------------------------------------------------------
// S1: ingest and rank reduction.
// ---------------------------------------------------------------------------
// Eight bytes, each 0 or 1, packed into eight bits (byte t -> bit t): the
// multiplier moves byte t's low bit to bit 56 + t, and no two partial products
// meet, so nothing carries.  The bytes are loaded little-endian (byte t of
// memory in bits 8t..8t+7), the order of both x86-64 and AArch64 Linux.
static inline uint32_t pack8(uint64_t b) { return (uint32_t)(((b & 0x0101010101010101ull) * 0x0102040810204080ull) >> 56); }

static int load_input(const uint8_t* gen, int n, int K, int field, Plan* p) {
    p->input.assign(K, Vec());
    uint64_t bad = 0;  // any symbol out of range
    for (int r = 0; r < K; r++) {
        Vec& v = p->input[r];
        memset(&v, 0, sizeof v);
        if (field == 2) {
            const uint8_t* xs = gen + (size_t)r * 2 * n;
            const uint8_t* zs = xs + n;
            int i = 0;
            for (; i + 8 <= n; i += 8) {
                uint64_t a, c;
                memcpy(&a, xs + i, 8);
                memcpy(&c, zs + i, 8);
                bad |= (a | c) & ~0x0101010101010101ull;
                v.x[i >> 5] |= pack8(a) << (i & 31);
                v.z[i >> 5] |= pack8(c) << (i & 31);
            }
            for (; i < n; i++) {
                bad |= (xs[i] | zs[i]) & ~1u;
                v.x[i >> 5] |= (uint32_t)(xs[i] & 1u) << (i & 31);
                v.z[i >> 5] |= (uint32_t)(zs[i] & 1u) << (i & 31);
            }
        } else {
            const uint8_t* s4 = gen + (size_t)r * n;
            for (int i = 0; i < n; i++) {
                bad |= s4[i] & ~3u;
                v.x[i >> 5] |= (uint32_t)(s4[i] & 1u) << (i & 31);
                v.z[i >> 5] |= (uint32_t)((s4[i] >> 1) & 1u) << (i & 31);
            }
        }
    }
    return bad ? P_EINVAL : P_OK;
}

// Keeps, in input order, the rows independent of the ones kept before them
// (over F2 for field 2, over F4 for field 4).
static void reduce_rank(Plan* p) {
    p->kept.clear();
    p->basis.clear();
    std::vector<Vec> ech;
    std::vector<int> piv;  // F2: bit index in [0, 2n) ; F4: coordinate
    for (int r = 0; r < p->K_in; r++) {
        Vec t = p->input[r];
        for (size_t e = 0; e < ech.size(); e++) {
            if (p->field == 2) {
                int q = piv[e];
                int b = q < p->n ? bit(t.x, q) : bit(t.z, q - p->n);
                if (b) vxor(t, ech[e]);
            } else {
                int c = proj(t, piv[e]);
                if (c) vxor(t, vscale(ech[e], c));  // ech rows have symbol 1 at their pivot
            }
        }
        if (vzero(t)) continue;
        int q = -1;
        if (p->field == 2) {
            for (int i = 0; i < 2 * p->n && q < 0; i++)
                if (i < p->n ? bit(t.x, i) : bit(t.z, i - p->n)) q = i;
        } else {
            for (int i = 0; i < p->n && q < 0; i++)
                if (proj(t, i)) q = i;
            t = vscale(t, f4_inv(proj(t, q)));
        }
        ech.push_back(t);
        piv.push_back(q);
        p->kept.push_back(r);
        p->basis.push_back(p->input[r]);
    }
    p->k_eff = (int)p->basis.size();
}

// ---------------------------------------------------------------------------
// S2: package diagonalization.
// ---------------------------------------------------------------------------

// Set of rows (bit i = row i) in NW 64-bit words.
template <int NW>
struct RowSet {
    uint64_t w[NW];
};
template <int NW>
static inline void rs_set(RowSet<NW>& s, int i) { s.w[i >> 6] |= 1ull << (i & 63); }
template <int NW>
static inline void rs_clear(RowSet<NW>& s, int i) { s.w[i >> 6] &= ~(1ull << (i & 63)); }
template <int NW>
static inline int rs_first(const RowSet<NW>& s) {  // lowest row, -1 if empty
    for (int t = 0; t < NW; t++)
        if (s.w[t]) return t * 64 + __builtin_ctzll(s.w[t]);
    return -1;
}
template <int NW>
static inline RowSet<NW> rs_and(const RowSet<NW>& a, const RowSet<NW>& b) {
    RowSet<NW> r;
    for (int t = 0; t < NW; t++) r.w[t] = a.w[t] & b.w[t];
    return r;
}
template <int NW>
static inline RowSet<NW> rs_andnot(const RowSet<NW>& a, const RowSet<NW>& b) {
    RowSet<NW> r;
    for (int t = 0; t < NW; t++) r.w[t] = a.w[t] & ~b.w[t];
    return r;
}
template <int NW>
static inline RowSet<NW> rs_or(const RowSet<NW>& a, const RowSet<NW>& b) {
    RowSet<NW> r;
    for (int t = 0; t < NW; t++) r.w[t] = a.w[t] | b.w[t];
    return r;
}
template <int NW>
static inline void rs_xor_into(RowSet<NW>& a, const RowSet<NW>& b) {
    for (int t = 0; t < NW; t++) a.w[t] ^= b.w[t];
}
template <int NW>
static inline bool rs_any(const RowSet<NW>& a) {
    uint64_t o = 0;
    for (int t = 0; t < NW; t++) o |= a.w[t];
    return o != 0;
}

// F2 (Sections 2.2-2.3 in F2 language).  Works on the qubits not used by an
// earlier matrix.  At each step it takes the unused qubit whose projections,
// over the rows not pivoted yet, span the most (rank 2 first, then rank 1,
// lowest index on ties):
//  * rank 2: two rows g, h with independent projections become a package
//    {g, h, g+h}; every other row gets the combination of g and h that clears
//    the qubit, so any sum that contains a package member is nonzero there.
//  * rank 1 (projections in {0, v}): a row g with projection v becomes a
//    one-element package.  Other rows may carry any projection; fix a nonzero
//    w != v and add g to every row whose projection is v or v+w.  Afterwards
//    all other rows lie in {0, w}, whose span never contains v or v+w, so any
//    sum containing g is nonzero at the qubit.
// Rows left without a pivot are free.  A later pivot only adds rows whose
// projection on earlier pivot qubits is already 0, so earlier packages keep
// their property.
// NW = words of a row set (k <= 64 NW).
template <int NW>
static void diag_f2_t(const Plan& p, const std::vector<int>& qorder, std::vector<char>& used, Gamma& G) {
    const int k = p.k_eff, n = p.n;
    std::vector<Vec> R = p.basis;
    std::vector<Coef> C(k);
    for (int i = 0; i < k; i++) {
        memset(&C[i], 0, sizeof(Coef));
        setb(C[i].p[0], i);
    }
    // Column view of R on the unused qubits: cx[q] (cz[q]) = rows with a 1 in
    // the x (z) plane at qubit q.  The projection of row i onto q is
    // (i in cx[q]) + 2 (i in cz[q]).  A qubit's column is not read once the
    // qubit is used, so only the unused ones are kept in step with the rows.
    uint32_t openq[DIST_MAXW] = {0};
    for (int q = 0; q < n; q++)
        if (!used[q]) setb(openq, q);
    std::vector<RowSet<NW>> cx(n), cz(n);
    memset(cx.data(), 0, n * sizeof(RowSet<NW>));
    memset(cz.data(), 0, n * sizeof(RowSet<NW>));
    for (int i = 0; i < k; i++)
        for (int w = 0; w < p.W; w++) {
            for (uint32_t m = R[i].x[w] & openq[w]; m; m &= m - 1) rs_set(cx[w * 32 + __builtin_ctz(m)], i);
            for (uint32_t m = R[i].z[w] & openq[w]; m; m &= m - 1) rs_set(cz[w * 32 + __builtin_ctz(m)], i);
        }
    RowSet<NW> unpiv;
    memset(&unpiv, 0, sizeof unpiv);
    for (int i = 0; i < k; i++) rs_set(unpiv, i);
    // rows with projection val (1, 2, 3) at q
    auto with_proj = [&](int q, int val) {
        return val == 1 ? rs_andnot(cx[q], cz[q]) : val == 2 ? rs_andnot(cz[q], cx[q]) : rs_and(cx[q], cz[q]);
    };
    // R[i] += v and C[i] += c (F2 coefficients: plane 0 only) for every row i
    // in S, at fixed widths, which the compiler vectorizes
    auto add_rows = [&](const RowSet<NW>& S, const Vec& v, const Coef& c) {
        for (int t = 0; t < NW; t++)
            for (uint64_t m = S.w[t]; m; m &= m - 1) {
                const int i = t * 64 + __builtin_ctzll(m);
                vxor(R[i], v);
                for (int w = 0; w < DIST_MAXCW; w++) C[i].p[0][w] ^= c.p[0][w];
            }
    };
    // the open columns after the rows of S took v
    auto add_cols = [&](const RowSet<NW>& S, const Vec& v) {
        for (int w = 0; w < p.W; w++) {
            for (uint32_t m = v.x[w] & openq[w]; m; m &= m - 1) rs_xor_into(cx[w * 32 + __builtin_ctz(m)], S);
            for (uint32_t m = v.z[w] & openq[w]; m; m &= m - 1) rs_xor_into(cz[w * 32 + __builtin_ctz(m)], S);
        }
    };
    std::vector<char> piv(k, 0);
    struct U { int kind, q, g, h; };
    std::vector<U> units;
    units.reserve(k);
    for (;;) {
        int best_q = -1, best_rank = 0;
        for (int t = 0; t < n; t++) {
            const int q = qorder[t];
            if (used[q]) continue;
            const RowSet<NW> a = rs_and(cx[q], unpiv), b = rs_and(cz[q], unpiv);
            const int nz = (int)rs_any(rs_andnot(a, b)) + (int)rs_any(rs_andnot(b, a)) + (int)rs_any(rs_and(a, b));
            const int rank = nz >= 2 ? 2 : nz;
            if (rank > best_rank) {
                best_rank = rank;
                best_q = q;
                if (rank == 2) break;
            }
        }
        if (best_rank == 0) break;
        const int q = best_q;
        // q is used from here on: its column is no longer updated
        used[q] = 1;
        openq[q >> 5] &= ~(1u << (q & 31));
        const RowSet<NW> live = rs_and(rs_or(cx[q], cz[q]), unpiv);  // unpivoted rows, nonzero at q
        const int g = rs_first(live);
        const int vg = proj(R[g], q);
        if (best_rank == 2) {
            const int h = rs_first(rs_andnot(live, with_proj(q, vg)));
            const int vh = proj(R[h], q);
            // rows with projection vg take g, vh take h, vg+vh take g+h
            RowSet<NW> Sg = with_proj(q, vg), Sh = with_proj(q, vh), Sgh = with_proj(q, vg ^ vh);
            rs_clear(Sg, g); rs_clear(Sg, h);
            rs_clear(Sh, g); rs_clear(Sh, h);
            rs_clear(Sgh, g); rs_clear(Sgh, h);
            add_cols(rs_or(Sg, Sgh), R[g]);
            add_cols(rs_or(Sh, Sgh), R[h]);
            Vec sv = R[g];
            vxor(sv, R[h]);
            Coef sc = C[g];
            for (int w = 0; w < DIST_MAXCW; w++) sc.p[0][w] ^= C[h].p[0][w];
            add_rows(Sg, R[g], C[g]);
            add_rows(Sh, R[h], C[h]);
            add_rows(Sgh, sv, sc);
            piv[g] = piv[h] = 1;
            rs_clear(unpiv, g);
            rs_clear(unpiv, h);
            units.push_back({UNIT_PACKAGE2, q, g, h});
        } else {
            const int v = vg;
            const int w = (v == 1) ? 2 : 1;  // smallest nonzero value other than v
            RowSet<NW> S = rs_or(with_proj(q, v), with_proj(q, v ^ w));
            rs_clear(S, g);
            add_cols(S, R[g]);
            add_rows(S, R[g], C[g]);
            piv[g] = 1;
            rs_clear(unpiv, g);
            units.push_back({UNIT_PACKAGE1, q, g, -1});
        }
        G.pivots.push_back(q);
    }
    for (int i = 0; i < k; i++)
        if (!piv[i]) units.push_back({UNIT_FREE, -1, i, -1});
    G.A.clear();
    G.B.clear();
    G.A.reserve(units.size());
    G.B.reserve(units.size());
    G.f = 0;
    G.npack = 0;
    for (const U& u : units) {
        Unit x;
        memset(&x, 0, sizeof x);
        x.kind = u.kind;
        x.qubit = u.q;
        x.rep[0] = R[u.g];
        x.coef[0] = C[u.g];
        if (u.kind == UNIT_PACKAGE2) {
            x.nrep = 3;
            x.rep[1] = R[u.h];
            x.coef[1] = C[u.h];
            x.rep[2] = R[u.g];
            vxor(x.rep[2], R[u.h]);
            x.coef[2] = C[u.g];
            cxor(x.coef[2], C[u.h]);
            G.A.push_back(x);
        } else {
            x.nrep = 1;
            G.B.push_back(x);
        }
        if (u.kind == UNIT_FREE) G.f++;
        else G.npack++;
    }
}

// diag_f2_t with row sets just wide enough for the k_eff rows
static void diag_f2(const Plan& p, const std::vector<int>& qorder, std::vector<char>& used, Gamma& G) {
    const int nw = (p.k_eff + 63) / 64;
    if (nw <= 1) diag_f2_t<1>(p, qorder, used, G);
    else if (nw == 2) diag_f2_t<2>(p, qorder, used, G);
    else if (nw == 3) diag_f2_t<3>(p, qorder, used, G);
    else diag_f2_t<4>(p, qorder, used, G);
}

// F4-linear codes (Section 2.3): reduced echelon form over F4 on the unused
// coordinates, lowest coordinate first.  Every row becomes a unit with the
// representatives g, alpha g, alpha^2 g; pivot rows are packages (weight >= 1
// on their pivot coordinate in any combination that uses them), the rest free.
static void diag_f4(const Plan& p, const std::vector<int>& qorder, std::vector<char>& used, Gamma& G) {
    const int k = p.k_eff, n = p.n;
    std::vector<Vec> R = p.basis;
    std::vector<Coef> C(k);
    for (int i = 0; i < k; i++) {
        memset(&C[i], 0, sizeof(Coef));
        setb(C[i].p[0], i);  // scalar 1 on basis row i
    }
    std::vector<char> piv(k, 0);
    std::vector<int> lst(k);
    std::vector<std::pair<int, int>> order;  // (row, qubit)
    int npiv = 0;
    for (int t = 0; t < n && npiv < k; t++) {
        const int q = qorder[t];
        if (used[q]) continue;
        int g = -1;
        for (int i = 0; i < k && g < 0; i++)
            if (!piv[i] && proj(R[i], q)) g = i;
        if (g < 0) continue;
        int inv = f4_inv(proj(R[g], q));
        R[g] = vscale(R[g], inv);
        C[g] = cscale(C[g], inv);
        // row i takes c R[g], c = its symbol at q (R[g] has symbol 1 there)
        Vec sv[4];
        Coef sc[4];
        for (int c = 1; c < 4; c++) {
            sv[c] = vscale(R[g], c);
            sc[c] = cscale(C[g], c);
        }
        int nl = 0;
        for (int i = 0; i < k; i++) {  // branch-free list of the rows to change
            lst[nl] = i;
            nl += (i != g) & (proj(R[i], q) != 0);
        }
        for (int t = 0; t < nl; t++) {
            const int i = lst[t], c = proj(R[i], q);
            vxor(R[i], sv[c]);
            cxor(C[i], sc[c]);
        }
        piv[g] = 1;
        npiv++;
        used[q] = 1;
        G.pivots.push_back(q);
        order.push_back({g, q});
    }
    for (int i = 0; i < k; i++)
        if (!piv[i]) order.push_back({i, -1});
    G.A.clear();
    G.B.clear();
    G.f = 0;
    G.npack = 0;
    for (auto& o : order) {
        Unit x;
        memset(&x, 0, sizeof x);
        x.kind = o.second >= 0 ? UNIT_PACKAGE2 : UNIT_FREE;
        x.qubit = o.second;
        x.nrep = 3;
        for (int e = 0; e < 3; e++) {
            x.rep[e] = vscale(R[o.first], e + 1);
            x.coef[e] = cscale(C[o.first], e + 1);
        }
        G.A.push_back(x);
        if (o.second >= 0) G.npack++;
        else G.f++;
    }
}

// Device tables of one matrix: qubits reordered so that the qubits that are
// NOT pivots of this matrix come first (they fill word 0 of each plane, the
// word the enumeration filters on), pivots after them.
static void build_device_tables(const Plan& p, Gamma& G) {
    G.tables_built = true;
    std::vector<char> isp(p.n, 0);
    for (int q : G.pivots) isp[q] = 1;
    G.perm.clear();
    for (int q = 0; q < p.n; q++)
        if (!isp[q]) G.perm.push_back(q);
    for (int q : G.pivots) G.perm.push_back(q);
    const int u = G.units(), W = p.W, CW = p.CW;
    G.dev_reps.assign((size_t)u * 3 * 2 * W, 0);
    G.dev_coefs.assign((size_t)u * 3 * 2 * CW, 0);
    // A package is nonzero at its pivot in every combination that uses it; if
    // the pivot sits outside word 0 this adds one to the word-0 lower bound.
    std::vector<int> pos_of(p.n, 0);
    for (int pos = 0; pos < p.n; pos++) pos_of[G.perm[pos]] = pos;
    G.dev_flags.assign((size_t)u, 0);
    for (int t = 0; t < u; t++) {
        const Unit& x = t < (int)G.A.size() ? G.A[t] : G.B[t - G.A.size()];
        if (x.qubit >= 0 && pos_of[x.qubit] >= 32) G.dev_flags[t] |= 1u;
        if (x.qubit >= 0 && pos_of[x.qubit] >= 64) G.dev_flags[t] |= 2u;
    }
    G.a_all = 3u;
    for (size_t t = 0; t < G.A.size(); t++) G.a_all &= G.dev_flags[t];
    G.dev_r0.assign(G.A.size() * 6, 0);
    G.dev_r1.assign(G.A.size() * 6, 0);
    // The qubit permutation as nibble tables: entry (N, v) is the 128-bit
    // image of value v in nibble N of a plane, so a plane maps with one lookup
    // per nibble.
    const int nnib = (p.n + 3) / 4;
    std::vector<uint64_t> img((size_t)nnib * 32);
    for (int N = 0; N < nnib; N++) {
        uint64_t* T = &img[(size_t)N * 32];
        T[0] = T[1] = 0;
        for (int v = 1; v < 16; v++) {
            const int q = N * 4 + __builtin_ctz((unsigned)v), prev = v & (v - 1);
            uint64_t lo = 0, hi = 0;
            if (q < p.n) {
                const int d = pos_of[q];
                if (d < 64) lo = 1ull << d;
                else hi = 1ull << (d - 64);
            }
            T[2 * v] = T[2 * prev] | lo;
            T[2 * v + 1] = T[2 * prev + 1] | hi;
        }
    }
    auto permute = [&](const uint32_t* src, uint32_t* dst) {
        uint64_t lo = 0, hi = 0;
        for (int N = 0; N < nnib; N++) {
            const unsigned v = (src[N >> 3] >> ((N & 7) * 4)) & 0xFu;
            lo |= img[((size_t)N * 16 + v) * 2];
            hi |= img[((size_t)N * 16 + v) * 2 + 1];
        }
        for (int w = 0; w < W; w++) dst[w] = (uint32_t)((w < 2 ? lo : hi) >> ((w & 1) * 32));
    };
    for (int t = 0; t < u; t++) {
        const Unit& x = t < (int)G.A.size() ? G.A[t] : G.B[t - G.A.size()];
        for (int e = 0; e < x.nrep; e++) {
            uint32_t* dx = &G.dev_reps[(((size_t)t * 3 + e) * 2 + 0) * W];
            uint32_t* dz = &G.dev_reps[(((size_t)t * 3 + e) * 2 + 1) * W];
            if (e == 2) {  // rep 2 = rep 0 + rep 1, and the permutation is linear
                for (int w = 0; w < W; w++) {
                    dx[w] = dx[w - 4 * W] ^ dx[w - 2 * W];
                    dz[w] = dz[w - 4 * W] ^ dz[w - 2 * W];
                }
            } else {
                permute(x.rep[e].x, dx);
                permute(x.rep[e].z, dz);
            }
            for (int c = 0; c < 2; c++)
                for (int w = 0; w < CW; w++)
                    G.dev_coefs[(((size_t)t * 3 + e) * 2 + c) * CW + w] = x.coef[e].p[c][w];
            if (t < (int)G.A.size()) {
                G.dev_r0[((size_t)t * 3 + e) * 2 + 0] = dx[0];
                G.dev_r0[((size_t)t * 3 + e) * 2 + 1] = dz[0];
                if (W >= 2) {
                    G.dev_r1[((size_t)t * 3 + e) * 2 + 0] = dx[1];
                    G.dev_r1[((size_t)t * 3 + e) * 2 + 1] = dz[1];
                }
            }
        }
    }
    // Level above which the one-word filter lets too many blocks through:
    // word 0 of a representative weighs mu +- sigma; a block of 81 codewords
    // slips through about 81 * Phi((thr - P - mu) / sigma) of the time, so
    // switch when thr - P > mu - 3.3 sigma.
    {
        double s1 = 0, s2 = 0, cnt = 0;
        for (size_t t = 0; t < G.A.size(); t++)
            for (int e = 0; e < 3; e++) {
                double w = __builtin_popcount(G.dev_r0[(t * 3 + e) * 2] | G.dev_r0[(t * 3 + e) * 2 + 1]);
                s1 += w;
                s2 += w * w;
                cnt += 1;
            }
        if (cnt > 1 && W >= 2) {
            double mu = s1 / cnt, var = std::max(0.0, s2 / cnt - mu * mu);
            G.t1 = (int)floor(mu - 3.3 * sqrt(var + 1.0));
        } else {
            G.t1 = 1 << 20;  // one word covers every qubit: never switch
        }
    }
}

static bool coef_outside(const Plan& p, const Coef& c) {
    if (p.n_stab == 0) return true;
    for (int w = 0; w < p.CW; w++)
        if ((c.p[0][w] | c.p[1][w]) & p.outside[w]) return true;
    return false;
}

// Lightest representative of any matrix (outside S if only_outside): its
// weight and a witness slot naming it.
static void lightest_rep(const Plan& p, bool only_outside, int* w_out, WitnessSlot* slot) {
    int best = DIST_WINF;
    memset(slot, 0, sizeof *slot);
    for (size_t g = 0; g < p.gammas.size(); g++) {
        const Gamma& G = p.gammas[g];
        for (int t = 0; t < G.units(); t++) {
            const Unit& x = t < (int)G.A.size() ? G.A[t] : G.B[t - G.A.size()];
            for (int e = 0; e < x.nrep; e++) {
                if (only_outside && !coef_outside(p, x.coef[e])) continue;
                int w = vec_weight(x.rep[e], p.W);
                if (w < best) {
                    best = w;
                    slot->claim = 1;
                    slot->gamma = (uint32_t)g;
                    slot->count = 1;
                    slot->weight = (uint32_t)w;
                    slot->unit[0] = (uint8_t)t;
                    slot->digit[0] = (uint8_t)e;
                }
            }
        }
    }
    *w_out = best;
}

// Number of codewords in round r of matrix g (F4: projective, first scalar 1).
double plan_round_count(const Plan& p, int g, int r) {
    const Gamma& G = p.gammas[g];
    const int a = (int)G.A.size(), b = (int)G.B.size();
    if (p.field == 4) return r >= 1 ? dbinom(a, r) * pow(3.0, r - 1) : 0.0;
    double s = 0;
    for (int i = std::max(0, r - b); i <= std::min(r, a); i++)
        s += dbinom(a, i) * pow(3.0, i) * dbinom(b, r - i);
    return s;
}

static int bound_for(const Plan& p, const std::vector<int>& J, int r, int jpos) {
    long L = 0;
    for (size_t t = 0; t < J.size(); t++) {
        const Gamma& G = p.gammas[J[t]];
        int rr = (int)t <= jpos ? r : r - 1;
        if (rr >= G.units()) return DIST_WINF;
        L += std::max(0, rr + 1 - G.f);
    }
    return (int)std::min<long>(L, DIST_WINF - 1);
}

int plan_lower_bound(const Plan& p, int r, int jpos) { return bound_for(p, p.J, r, jpos); }

int plan_initial_bound(const Plan& p) { return std::max(1, bound_for(p, p.J, 0, (int)p.J.size())); }

static std::atomic<int> g_gamma_limit{0};
int plan_gamma_limit() { return g_gamma_limit.load(); }
void plan_set_gamma_limit(int m) { g_gamma_limit.store(std::max(0, std::min(m, DIST_MAXGAMMA))); }

// Choice of J: among the matrices sorted by free rows, the prefix whose
// estimated work to lift the bound to d_est is smallest.  Any nonempty J is
// correct; this only decides speed.
static double choose_J(Plan* p) {
    std::vector<int> cand;
    for (size_t g = 0; g < p->gammas.size(); g++) cand.push_back((int)g);
    std::stable_sort(cand.begin(), cand.end(),
                     [&](int a, int b) { return p->gammas[a].f < p->gammas[b].f; });
    double best = INFINITY;
    std::vector<int> bestJ;
    // Every prefix sums the same round counts: each (matrix, round) is
    // computed once, as plan_round_count does, from binomials and powers of 3
    // computed once each (the same values, summed in the same order).
    std::vector<std::vector<double>> cnt(p->gammas.size()), ca(p->gammas.size()), cb(p->gammas.size());
    std::vector<double> p3;
    auto count = [&](int g, int r) {
        std::vector<double>& v = cnt[g];
        while ((int)v.size() <= r) v.push_back(-1.0);
        if (v[r] >= 0) return v[r];
        const Gamma& G = p->gammas[g];
        const int a = (int)G.A.size(), b = (int)G.B.size();
        auto binom = [](std::vector<double>& t, int m, int i) {  // C(m, i), i <= m
            if (t.empty()) t.assign(m + 1, -1.0);
            if (t[i] < 0) t[i] = dbinom(m, i);
            return t[i];
        };
        while ((int)p3.size() <= r) p3.push_back(pow(3.0, (double)p3.size()));
        double s = 0;
        if (p->field == 4) {
            s = r >= 1 ? (r <= a ? binom(ca[g], a, r) : 0.0) * p3[r - 1] : 0.0;
        } else {
            for (int i = std::max(0, r - b); i <= std::min(r, a); i++)
                s += binom(ca[g], a, i) * p3[i] * binom(cb[g], b, r - i);
        }
        v[r] = s;
        return s;
    };
    const int limit = plan_gamma_limit();
    const size_t mmax = limit > 0 ? std::min(cand.size(), (size_t)limit) : cand.size();
    for (size_t m = 1; m <= mmax; m++) {
        std::vector<int> J(cand.begin(), cand.begin() + m);
        double work = 0;
        for (int r = 1; r <= DIST_MAXU; r++) {
            for (size_t t = 0; t < J.size(); t++) {
                work += count(J[t], r);
                if (bound_for(*p, J, r, (int)t) >= p->d_est) goto done;
            }
        }
    done:
        if (work < best) {
            best = work;
            bestJ = J;
        }
    }
    p->J = bestJ;
    return best;
}

// Estimated work (codewords) above which plan_build tries other qubit
// orders, and how many: a search trial costs about one diagonalization (tens
// of microseconds), a round it saves often tens of millions of codewords.
static constexpr double kSearchWork = 5e8;
static std::atomic<int> g_plan_search_trials{8};

int plan_search_trials() { return g_plan_search_trials.load(); }
void plan_set_search_trials(int t) { g_plan_search_trials.store(std::max(0, std::min(t, 256))); }

// Does some matrix of J have free rows (a round that adds less than 1 to L)?
static bool free_rows_in_J(const Plan& p) {
    for (int g : p.J)
        if (p.gammas[g].f > 0) return true;
    return false;
}

// The codeword a seed slot names (a representative, or the plan's seed).
static void slot_codeword(const Plan& p, const WitnessSlot& s, Vec* v, Coef* k) {
    if (s.gamma == DIST_SEED_GAMMA) {
        *v = p.seed_vec;
        *k = p.seed_coef;
        return;
    }
    const Gamma& G = p.gammas[s.gamma];
    const Unit& x = s.unit[0] < G.A.size() ? G.A[s.unit[0]] : G.B[s.unit[0] - G.A.size()];
    *v = x.rep[s.digit[0]];
    *k = x.coef[s.digit[0]];
}

// S2 with the unused qubits considered in qorder, then the seed U, d_est
// (d_random capped by the seed) and J (no device tables yet).  A known codeword lighter than every
// representative of this diagonalization becomes the seed.  *work = the
// estimated codewords to lift the bound to d_est.
// Expected number of nonzero codewords of weight <= w in a random code of
// the same size: 2^(K2 - 2n) * sum_v C(n, v) 3^v.  The estimate of d is the
// first w where it reaches 1 (n if none).
static int random_code_d(const Plan& p) {
    const int n = p.n, K2 = p.field == 2 ? p.k_eff : 2 * p.k_eff;
    double acc = 0;
    for (int w = 1; w <= n; w++) {
        acc += dbinom(n, w) * pow(3.0, w);
        if (log2(acc) + K2 - 2.0 * n >= 0) return w;
    }
    return n;
}

// S2 proper: the generator matrices of p's basis on disjoint qubit sets,
// visiting the qubits in qorder.
static int build_matrices(Plan* p, const std::vector<int>& qorder) {
    const int n = p->n, field = p->field;
    p->gammas.clear();
    std::vector<char> used(n, 0);
    // qubits where some basis row is nonzero: a matrix needs an unused one
    Vec support;
    memset(&support, 0, sizeof support);
    for (const Vec& b : p->basis)
        for (int w = 0; w < p->W; w++) support.x[w] |= b.x[w] | b.z[w];
    for (int j = 0; j < DIST_MAXGAMMA; j++) {
        bool open = false;
        for (int q = 0; q < n && !open; q++) open = !used[q] && bit(support.x, q);
        if (!open) break;
        Gamma G;
        std::vector<char> u2 = used;
        if (field == 2) diag_f2(*p, qorder, u2, G);
        else diag_f4(*p, qorder, u2, G);
        if (G.npack == 0) break;
        if (G.A.size() > 255 || G.units() > DIST_MAXU) return P_ERANGE;
        used = u2;
        p->gammas.push_back(std::move(G));
    }
    if (p->gammas.empty()) return P_EZERO;
    return P_OK;
}

// The rest of a plan once its matrices are built: the seed of the upper
// bound (the lightest representative, or a lighter codeword known from
// another plan), the estimate of d and the choice of J.
static int finish_plan(Plan* p, int d_random, double* work, int known_w = DIST_WINF, const Vec* known_v = nullptr,
                       const Coef* known_k = nullptr) {
    // The lightest representative is a codeword: it seeds the upper bound.
    p->u0 = DIST_WINF;
    lightest_rep(*p, false, &p->u0, &p->u0_slot);
    if (known_v && known_w < p->u0) {
        p->u0 = known_w;
        memset(&p->u0_slot, 0, sizeof p->u0_slot);
        p->u0_slot.claim = 1;
        p->u0_slot.gamma = DIST_SEED_GAMMA;
        p->u0_slot.weight = (uint32_t)known_w;
        p->seed_vec = *known_v;
        p->seed_coef = *known_k;
    }
    p->d_est = std::max(1, std::min(d_random, p->u0));
    *work = choose_J(p);
    return P_OK;
}

static int diagonalize(Plan* p, const std::vector<int>& qorder, int d_random, double* work) {
    const int rc = build_matrices(p, qorder);
    return rc ? rc : finish_plan(p, d_random, work);
}

namespace {

// One persistent helper thread, so that plan_build can build the first
// search trial's matrices while the index-order plan is built (a thread
// started per call would cost about as much as the overlap saves).  A caller
// that finds it busy does the work itself.  Waking a sleeping thread takes
// from a few to tens of microseconds, as long as the job itself, so both
// sides spin for a short while before they sleep: the helper for kIdleSpin
// after each job (the next plan_build of a stream of codes then finds it
// awake), the caller for kWaitSpin in wait().
class Helper {
   public:
    bool try_run(std::function<void()> job) {
        // a child process made by fork() has no helper thread (and its lock
        // may have been held at the fork): the caller does the work
        if (getpid() != owner_) return false;
        std::lock_guard<std::mutex> lk(mu_);
        if (busy_.load(std::memory_order_relaxed)) return false;
        job_ = std::move(job);
        busy_.store(true, std::memory_order_release);
        pending_.store(true, std::memory_order_release);
        cv_.notify_one();
        return true;
    }
    void wait() {
        if (spin_until([this] { return !busy_.load(std::memory_order_acquire); }, kWaitSpin)) return;
        std::unique_lock<std::mutex> lk(mu_);
        done_.wait(lk, [this] { return !busy_.load(std::memory_order_acquire); });
    }
    static Helper& get() {
        static Helper* h = new Helper();  // never destroyed: its thread runs until exit
        return *h;
    }

   private:
    static constexpr double kIdleSpin = 2e-3, kWaitSpin = 2e-3;  // seconds
    // Polls pred for up to `seconds`; true if it held.
    template <class Pred>
    static bool spin_until(Pred pred, double seconds) {
        const auto t0 = std::chrono::steady_clock::now();
        for (unsigned it = 0;; it++) {
            if (pred()) return true;
            if ((it & 255u) == 255u &&
                std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > seconds)
                return false;
        }
    }
    Helper() : owner_(getpid()) { std::thread([this] { loop(); }).detach(); }
    void loop() {
        for (;;) {
            spin_until([this] { return pending_.load(std::memory_order_acquire); }, kIdleSpin);
            std::function<void()> job;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [this] { return pending_.load(std::memory_order_relaxed); });
                pending_.store(false, std::memory_order_relaxed);
                job = std::move(job_);
                job_ = nullptr;
            }
            job();
            {
                std::lock_guard<std::mutex> lk(mu_);
                busy_.store(false, std::memory_order_release);
            }
            done_.notify_all();
        }
    }
    std::mutex mu_;
    std::condition_variable cv_, done_;
    std::function<void()> job_;
    std::atomic<bool> busy_{false}, pending_{false};
    const pid_t owner_;
};

// Fisher-Yates with xorshift64* on qorder, advancing the generator x.
void shuffle_order(std::vector<int>& qorder, uint64_t& x) {
    for (int q = (int)qorder.size() - 1; q > 0; q--) {
        x ^= x >> 12;
        x ^= x << 25;
        x ^= x >> 27;
        const int j = (int)(((x * 0x2545F4914F6CDD1Dull) >> 33) % (uint64_t)(q + 1));
        std::swap(qorder[q], qorder[j]);
    }
}

// A plan on p's basis with no matrices yet.
Plan empty_like(const Plan& p) {
    Plan alt;
    alt.n = p.n;
    alt.field = p.field;
    alt.K_in = p.K_in;
    alt.W = p.W;
    alt.CW = p.CW;
    alt.k_eff = p.k_eff;
    alt.input = p.input;
    alt.kept = p.kept;
    alt.basis = p.basis;
    return alt;
}

// Codes from this size on (qubits) build the first search trial's matrices
// beside the index-order plan: large codes are where the search runs.
constexpr int kSpeculateN = 48;

}  // namespace

// Independence of a few rows over F2 (elimination on the lowest set bit).
static bool rows_independent(std::vector<Vec> rows) {
    std::vector<int> piv;
    for (size_t i = 0; i < rows.size(); i++) {
        Vec& t = rows[i];
        for (size_t e = 0; e < i; e++) {
            const int q = piv[e];
            const int b = q < DIST_MAXN ? bit(t.x, q) : bit(t.z, q - DIST_MAXN);
            if (b) vxor(t, rows[e]);
        }
        int q = -1;
        for (int w = 0; w < DIST_MAXW && q < 0; w++)
            if (t.x[w]) q = w * 32 + __builtin_ctz(t.x[w]);
        for (int w = 0; w < DIST_MAXW && q < 0; w++)
            if (t.z[w]) q = DIST_MAXN + w * 32 + __builtin_ctz(t.z[w]);
        if (q < 0) return false;
        piv.push_back(q);
    }
    return true;
}

// Returned by plan_from_basis when rows it took as independent are not.
static constexpr int kDependent = 1;

static int plan_from_basis(Plan* p, bool assume_independent);

int plan_build(const uint8_t* gen, int n, int K, int field, Plan* p) {
    if (!gen || n < 1 || n > DIST_MAXN || K < 1) return P_EINVAL;
    if (field != 2 && field != 4) return P_EINVAL;
    if ((field == 2 ? K : 2 * K) > DIST_MAXK) return P_EINVAL;
    if (field == 2 && K > 2 * n) { /* dependent by counting; allowed, reduced below */ }
    *p = Plan();
    p->n = n;
    p->field = field;
    p->K_in = K;
    p->W = (n + 31) / 32;
    int rc = load_input(gen, n, K, field, p);
    if (rc) return rc;
    // Over F2 the rows are first taken as they are: the diagonalization shows
    // whether they are independent (below), and only if they are not does
    // the plan start again from the rows the elimination keeps.  Both ways
    // give the same plan for independent rows.
    if (field == 2 && K <= 2 * n) {
        rc = plan_from_basis(p, true);
        if (rc != kDependent) return rc;
        Plan q;
        q.n = n;
        q.field = field;
        q.K_in = K;
        q.W = p->W;
        q.input = std::move(p->input);
        *p = std::move(q);
    }
    return plan_from_basis(p, false);
}

// plan_build from the loaded input rows on: the basis (all rows, or the
// independent ones in input order), S2 with the qubit-order search, tables.
static int plan_from_basis(Plan* p, bool assume_independent) {
    const int n = p->n, K = p->K_in;
    int rc;
    if (assume_independent) {
        p->kept.resize(K);
        for (int r = 0; r < K; r++) p->kept[r] = r;
        p->basis = p->input;
        p->k_eff = K;
    } else {
        reduce_rank(p);
    }
    if (p->k_eff == 0) return P_EZERO;
    p->CW = (p->k_eff + 31) / 32;

    // S2 with the qubits in index order; for a code whose estimated work is
    // large, also with a few seeded random qubit orders (information sets can
    // be chosen freely: only speed depends on them), keeping the plan with
    // the least estimated work.  A later matrix on the leftover qubits often
    // has free rows, and each free row costs a whole round; another order
    // can leave it none.
    std::vector<int> qorder(n);
    for (int q = 0; q < n; q++) qorder[q] = q;
    double work = 0;
    const int d_random = random_code_d(*p);
    const int trials = plan_search_trials();
    // The first trial's qubit order, and its matrices built on the helper
    // thread while this one plans the index order (its matrices do not
    // depend on that plan; what does is done below, in the same order as
    // without the helper, so the result is the same).
    uint64_t x = 0x9E3779B97F4A7C15ull ^ (uint64_t)n * 0x100000001B3ull ^ (uint64_t)K;
    std::vector<int> qorder1 = qorder;
    uint64_t x1 = x;
    shuffle_order(qorder1, x1);
    Plan alt1;
    int rc1 = P_EINVAL;
    bool spec = false;
    if (trials > 0 && n >= kSpeculateN) {
        alt1 = empty_like(*p);
        // with its device tables: when the trial is needed it is usually kept
        spec = Helper::get().try_run([&alt1, &qorder1, &rc1] {
            rc1 = build_matrices(&alt1, qorder1);
            if (rc1 == P_OK)
                for (Gamma& G : alt1.gammas) build_device_tables(alt1, G);
        });
    }
    rc = diagonalize(p, qorder, d_random, &work);
    if (spec) Helper::get().wait();
    if (assume_independent) {
        // A combination that uses a package member is nonzero at that
        // package's pivot (Section 2.2), so the rows are independent exactly
        // when the first matrix's free rows are.
        if (rc != P_OK) return kDependent;
        std::vector<Vec> free_rows;
        for (const Unit& x : p->gammas[0].B)
            if (x.kind == UNIT_FREE) free_rows.push_back(x.rep[0]);
        if (!rows_independent(free_rows)) return kDependent;
    }
    if (rc) return rc;
    if (trials > 0 && work > kSearchWork && free_rows_in_J(*p)) {
        // the lightest codeword seen so far is an upper bound for every plan
        int kw = p->u0;
        Vec kv;
        Coef kk;
        slot_codeword(*p, p->u0_slot, &kv, &kk);
        for (int t = 0; t < trials && free_rows_in_J(*p); t++) {
            Plan alt;
            int rcm;
            if (t == 0) {
                qorder = qorder1;
                x = x1;
                if (spec) {
                    alt = std::move(alt1);
                    rcm = rc1;
                } else {
                    alt = empty_like(*p);
                    rcm = build_matrices(&alt, qorder);
                }
            } else {
                shuffle_order(qorder, x);
                alt = empty_like(*p);
                rcm = build_matrices(&alt, qorder);
            }
            double w2 = 0;
            if (rcm != P_OK || finish_plan(&alt, d_random, &w2, kw, &kv, &kk) != P_OK) continue;
            if (alt.u0 < kw) {  // a lighter representative: the new best seed
                kw = alt.u0;
                slot_codeword(alt, alt.u0_slot, &kv, &kk);
            }
            if (w2 < work) {
                work = w2;
                *p = std::move(alt);
            }
        }
    }
    for (Gamma& G : p->gammas)
        if (!G.tables_built) build_device_tables(*p, G);

    size_t off = 0;
    for (Gamma& G : p->gammas) {
        G.rep_off = (uint32_t)off;
        off += G.dev_reps.size();
        G.coef_off = (uint32_t)off;
        off += G.dev_coefs.size();
        G.flag_off = (uint32_t)off;
        off += G.dev_flags.size();
        off = (off + 1) & ~(size_t)1;
        G.r0_off = (uint32_t)off;
        off += G.dev_r0.size();
        G.r1_off = (uint32_t)off;
        off += G.dev_r1.size();
        off = (off + 3) & ~(size_t)3;
    }
    p->tables.assign(off, 0);
    for (const Gamma& G : p->gammas) {
        std::copy(G.dev_reps.begin(), G.dev_reps.end(), p->tables.begin() + G.rep_off);
        std::copy(G.dev_coefs.begin(), G.dev_coefs.end(), p->tables.begin() + G.coef_off);
        std::copy(G.dev_flags.begin(), G.dev_flags.end(), p->tables.begin() + G.flag_off);
        std::copy(G.dev_r0.begin(), G.dev_r0.end(), p->tables.begin() + G.r0_off);
        std::copy(G.dev_r1.begin(), G.dev_r1.end(), p->tables.begin() + G.r1_off);
    }
    p->u0_excl = p->u0;
    p->u0_excl_slot = p->u0_slot;
    return P_OK;
}

int plan_set_exclude(Plan* p, int n_stab) {
    if (n_stab < 0 || n_stab > p->K_in) return P_EINVAL;
    p->n_stab = n_stab;
    p->s_rank = 0;
    for (int r : p->kept)
        if (r < n_stab) p->s_rank++;
    memset(p->outside, 0, sizeof p->outside);
    if (n_stab > 0)
        for (int i = p->s_rank; i < p->k_eff; i++) setb(p->outside, i);
    // lightest representative outside S: an upper bound on the excluded minimum
    p->u0_excl = p->u0;
    p->u0_excl_slot = p->u0_slot;
    if (n_stab > 0) {
        p->u0_excl = DIST_WINF;
        lightest_rep(*p, true, &p->u0_excl, &p->u0_excl_slot);
        if (p->u0_slot.gamma == DIST_SEED_GAMMA && p->u0 < p->u0_excl && coef_outside(*p, p->seed_coef)) {
            p->u0_excl = p->u0;
            p->u0_excl_slot = p->u0_slot;
        }
    }
    if (n_stab > 0 && p->s_rank == p->k_eff) return P_EZERO;
    return P_OK;
}

// Cuts the raw segments of a planned launch into warp-chunks for
// target_warps resident warps (see plan_launch) and places the segment table
// in shared memory.
// Cost of a codeword on the generic path (full weights from scratch) in
// fast-path codewords, for sizing chunks.
static constexpr double kGenericCost = 32.0;

// Fewest chunks per resident warp that the lane floor may leave a fast-path
// segment: with about one chunk per warp the warps that drew a chunk late
// leave the others idle for most of a chunk, and with very small chunks the
// lane set-up dominates.  Measured on a launch whose last step has 376,992
// subsets of 243 codewords for 2432 warps: four subsets per lane (the floor
// alone) 0.0764 ms, three 0.0734 ms, two (this setting) 0.0724 ms, one
// 0.0800 ms.
static constexpr double kSpreadChunks = 2.0;

static void chunk_launch(LaunchPlan* lp, int target_warps) {
    // Chunks: each segment is cut into about chunks_per_warp (default 6)
    // warp-chunks per resident warp, so that every segment spreads over the
    // whole GPU and the tail is short; a lane chunk holds at most
    // 2^lane_cap_log2 (default 2^14, about a quarter of a millisecond for a
    // warp) codewords so that stop requests and time budgets are seen soon.
    // A segment on the
    // fast path gets at least 2^lane_floor_log2 codewords per lane, so that it
    // is not cut finer than the per-lane set-up (unranking the start subset,
    // fetching the chunk) is worth -- but never fewer chunks than
    // kSpreadChunks per resident warp: the early, small steps are where the
    // lighter codewords that lower U come from, and they must still spread
    // over the whole GPU.
    // Generic-path segments cost tens of times more per codeword and keep
    // the plain split, so that they never become the critical path.
    // Outside the launch's last step a fast-path lane chunk holds at least
    // eight subsets: a chunk costs about as much to start (claim, segment
    // search, unranking) as a few subsets of 81 to 243 codewords cost to
    // walk, and later steps keep every warp busy meanwhile.
    //
    // A large segment ends in smaller chunks: the work of one wave of
    // full-size chunks (one per resident warp) is cut into quarter-size ones,
    // which run while the last full-size chunks finish.  Whichever step turns
    // out to be the last one needed, warps then run out of work at nearly the
    // same time instead of waiting for the last full-size chunks.
    unsigned long long chunks = 0;
    const Tuning tun = tuning_get();
    const unsigned long long tw = (unsigned long long)std::max(1, target_warps);
    const std::vector<SegDesc>& raw = lp->raw_segs;
    std::vector<SegDesc> out;
    out.reserve(raw.size() + 16);
    std::vector<int> first_piece(raw.size());
    size_t spare = DIST_MAXSEG - raw.size();  // room for tail pieces
    for (size_t t = 0; t < raw.size(); t++) {
        SegDesc sd = raw[t];
        const double seg_cw = (double)sd.NA * (double)sd.NB * (double)sd.codes;
        double per_lane = seg_cw / (32.0 * (double)tw * (double)tun.chunks_per_warp);
        if (DIST_FAST_PATH((int)sd.i, lp->proj)) {
            const double spread = seg_cw / (32.0 * (double)tw * kSpreadChunks);
            per_lane = std::max(per_lane, std::min((double)(1u << tun.lane_floor_log2), spread));
            per_lane = std::min(per_lane, (double)(1u << tun.lane_cap_log2));
        } else {
            // a generic-path codeword costs tens of fast-path ones: cap its
            // lanes lower, so that a chunk lasts about as long either way
            per_lane = std::min(per_lane, (double)(1u << tun.lane_cap_log2) / kGenericCost);
        }
        double spl_d = per_lane / (double)sd.codes;
        if (DIST_FAST_PATH((int)sd.i, lp->proj) && (int)t < lp->raw_step_seg0.back() && spl_d < 8.0)
            spl_d = 8.0;
        unsigned long long spl = spl_d < 1.0 ? 1ull : (unsigned long long)spl_d;
        if (spl > (1ull << 30)) spl = 1ull << 30;
        const unsigned long long R = sd.rank1 - sd.rank0;
        first_piece[t] = (int)out.size();
        unsigned long long tail = 0;
        if (spl >= 4 && (R + 32 * spl - 1) / (32 * spl) >= 2 * tw && spare > 0) {
            tail = std::min(R / 2, tw * 32 * spl);
            --spare;
        }
        sd.spl = (uint32_t)spl;
        sd.chunk_base = chunks;
        sd.rank1 = sd.rank0 + (R - tail);
        chunks += (R - tail + 32 * spl - 1) / (32 * spl);
        out.push_back(sd);
        if (tail) {
            sd.spl = (uint32_t)(spl / 4);
            sd.chunk_base = chunks;
            sd.rank0 = sd.rank1;
            sd.rank1 = sd.rank0 + tail;
            chunks += (tail + 32 * (spl / 4) - 1) / (32 * (spl / 4));
            out.push_back(sd);
        }
    }
    lp->step_seg0 = lp->raw_step_seg0;
    for (int& s0 : lp->step_seg0) s0 = s0 < (int)first_piece.size() ? first_piece[s0] : (int)out.size();
    lp->segs.swap(out);
    lp->nchunks = chunks;
    lp->step_chunk0.clear();
    for (size_t s = 0; s < lp->step_r.size(); s++) {
        const int s0 = lp->step_seg0[s];
        lp->step_chunk0.push_back(s0 < (int)lp->segs.size() ? lp->segs[s0].chunk_base : chunks);
    }
    lp->s_words = lp->s_segs + (uint32_t)(lp->segs.size() * sizeof(SegDesc) / 4);
}

int plan_launch(const Plan& p, int r, int jpos, int L_prev, int U_bound, int target_warps,
                double max_codewords, LaunchPlan* lp) {
    *lp = LaunchPlan();
    lp->W = p.W;
    lp->CW = p.CW;
    lp->proj = p.field == 4 ? 1 : 0;
    lp->exclude = p.n_stab > 0 ? 1 : 0;
    std::vector<int> gslot(p.gammas.size(), -1);
    int L = L_prev, maxrow = 1, maxr = 1;
    double total = 0;
    std::vector<double> seg_cw;
    // room for a typical launch, so that the vectors grow without copies
    seg_cw.reserve(64);
    lp->segs.reserve(64);
    lp->g.reserve(p.J.size());
    lp->step_r.reserve(32);
    lp->step_jpos.reserve(32);
    lp->step_L_before.reserve(32);
    lp->step_seg0.reserve(32);
    for (;;) {
        if (r > DIST_MAXR) {
            if (lp->step_r.empty()) return P_ERANGE;
            break;
        }
        if (!lp->step_r.empty() && (L >= U_bound || total >= max_codewords)) break;
        const int g = p.J[jpos];
        const Gamma& G = p.gammas[g];
        const int a = (int)G.A.size(), b = (int)G.B.size();
        int imin = std::max(0, r - b), imax = std::min(r, a);
        if (lp->proj) imin = std::max(imin, 1);
        if (imax >= imin && lp->segs.size() + (imax - imin + 1) > DIST_MAXSEG) {
            if (lp->step_r.empty()) return P_ERANGE;
            break;
        }
        lp->step_seg0.push_back((int)lp->segs.size());
        if (gslot[g] < 0) {
            gslot[g] = (int)lp->g.size();
            GammaDesc d;
            memset(&d, 0, sizeof d);
            d.rep_off = G.rep_off;
            d.coef_off = G.coef_off;
            d.flag_off = G.flag_off;
            d.r0_off = G.r0_off;
            d.r1_off = G.r1_off;
            d.t1 = G.t1;
            d.a_all = G.a_all;
            d.a = (uint16_t)a;
            d.b = (uint16_t)b;
            d.gamma = g;
            lp->g.push_back(d);
        }
        for (int i = imin; i <= imax; i++) {
            unsigned long long NA = ubinom(a, i), NB = ubinom(b, r - i);
            unsigned long long codes = lp->proj ? upow3(i - 1) : upow3(i);
            if (NA == 0 || NB == 0) continue;
            if (NA == ~0ull || NB == ~0ull || codes == ~0ull || (((unsigned __int128)NA * NB) >> 62)) {
                // too many combinations to index: stop the plan before this step
                if (lp->step_r.empty()) return P_ERANGE;
                lp->segs.resize(lp->step_seg0.back());
                seg_cw.resize(lp->segs.size());
                lp->step_seg0.pop_back();
                goto planned;
            }
            SegDesc sd;
            memset(&sd, 0, sizeof sd);
            sd.NA = NA;
            sd.NB = NB;
            sd.rank0 = 0;
            sd.rank1 = NA * NB;
            sd.codes = codes;
            sd.i = (uint32_t)i;
            sd.g = (uint16_t)gslot[g];
            sd.r = (uint16_t)r;
            sd.L_before = L;
            lp->segs.push_back(sd);
            const double cw = (double)NA * (double)NB * (double)codes;
            seg_cw.push_back(cw);
            total += cw;
        }
        lp->step_r.push_back(r);
        lp->step_jpos.push_back(jpos);
        lp->step_L_before.push_back(L);
        maxrow = std::max(maxrow, std::max(a, b));
        maxr = std::max(maxr, r);
        L = plan_lower_bound(p, r, jpos);
        if (++jpos == (int)p.J.size()) {
            jpos = 0;
            ++r;
        }
        if (L == (int)DIST_WINF) break;  // this step finished a complete enumeration
    }
planned:
    lp->next_r = r;
    lp->next_jpos = jpos;
    total = 0;
    for (double cw : seg_cw) total += cw;
    lp->codewords = total;
    lp->raw_segs = lp->segs;
    lp->raw_step_seg0 = lp->step_seg0;
    // Shared memory (32-bit words): representatives of every matrix, their
    // word-0 tables, the binomials the launch can need, then the segment
    // table (placed by chunk_launch).
    uint32_t off = 0;
    for (GammaDesc& d : lp->g) {
        d.s_rep = off;
        off += (uint32_t)(d.a + d.b) * 6u * (uint32_t)p.W;
    }
    for (GammaDesc& d : lp->g) {
        off = (off + 1) & ~1u;
        d.s_r0 = off;
        off += (uint32_t)d.a * 6u;
        d.s_r1 = off;
        off += (uint32_t)d.a * 6u;
    }
    for (GammaDesc& d : lp->g) {
        d.s_flag = off;
        off += (uint32_t)(d.a + d.b);
    }
    off = (off + 1) & ~1u;
    lp->s_binom = off;
    lp->brows = maxrow + 1;
    lp->bcols = maxr + 1;
    off += (uint32_t)(lp->brows * lp->bcols) * 2u;
    lp->s_segs = off;
    chunk_launch(lp, target_warps);
    return P_OK;
}

int plan_rechunk(LaunchPlan* lp, int target_warps) {
    chunk_launch(lp, target_warps);
    return P_OK;
}

SliceVerdict plan_after_slice(const Plan& p, const LaunchPlan& lp, uint32_t U, unsigned long long next) {
    SliceVerdict v{SLICE_CONTINUE, 0, 0};
    if (next > lp.nchunks) next = lp.nchunks;
    for (size_t s = 0; s < lp.step_r.size(); s++) {
        if (U != DIST_WINF && (int)U <= lp.step_L_before[s]) {
            // every step before s is complete once s has started
            if (next >= lp.step_chunk0[s]) {
                v.kind = SLICE_CERTIFIED;
                v.L = lp.step_L_before[s];
            }
            return v;
        }
        const unsigned long long end = s + 1 < lp.step_r.size() ? lp.step_chunk0[s + 1] : lp.nchunks;
        if (next >= end) v.last_round = lp.step_r[s];
    }
    if (next < lp.nchunks) return v;
    const int La = plan_lower_bound(p, lp.step_r.back(), lp.step_jpos.back());
    v.L = La;
    v.kind = (La == (int)DIST_WINF || (U != DIST_WINF && La >= (int)U)) ? SLICE_CERTIFIED : SLICE_REPLAN;
    return v;
}

int plan_partial_bound(const Plan& p, const LaunchPlan& lp, unsigned long long next) {
    if (next > lp.nchunks) next = lp.nchunks;
    for (size_t s = 0; s < lp.step_r.size(); s++) {
        const unsigned long long end = s + 1 < lp.step_r.size() ? lp.step_chunk0[s + 1] : lp.nchunks;
        if (next < end) return lp.step_L_before[s];
    }
    return lp.step_r.empty() ? 1 : plan_lower_bound(p, lp.step_r.back(), lp.step_jpos.back());
}

void plan_params(const Plan& p, const LaunchPlan& lp, EnumParams* ep) {
    memset(ep, 0, sizeof *ep);
    for (int w = 0; w < DIST_MAXCW; w++) ep->outside[w] = p.outside[w];
    ep->W = lp.W;
    ep->CW = lp.CW;
    ep->proj = lp.proj;
    ep->exclude = lp.exclude;
    ep->ng = (int)lp.g.size();
    for (size_t t = 0; t < lp.g.size(); t++) ep->g[t] = lp.g[t];
    ep->nseg = (int)lp.segs.size();
    ep->brows = lp.brows;
    ep->bcols = lp.bcols;
    ep->s_binom = lp.s_binom;
    ep->s_segs = lp.s_segs;
    ep->s_words = lp.s_words;
    ep->nchunks = lp.nchunks;
}

int plan_decode_coef(const Plan& p, const Coef& k, int weight, uint8_t* witness, uint8_t* coeffs,
                     const Vec* expect) {
    if (!coef_outside(p, k)) return P_EINVAL;
    // the codeword the coefficients build from the input rows
    Vec c;
    memset(&c, 0, sizeof c);
    for (int i = 0; i < p.k_eff; i++) {
        int sym = bit(k.p[0], i) | (bit(k.p[1], i) << 1);
        if (sym) vxor(c, p.field == 2 ? p.input[p.kept[i]] : vscale(p.input[p.kept[i]], sym));
    }
    if (weight != vec_weight(c, p.W)) return P_EINVAL;
    if (expect)
        for (int w = 0; w < DIST_MAXW; w++)
            if (expect->x[w] != c.x[w] || expect->z[w] != c.z[w]) return P_EINVAL;
    if (witness) {
        for (int i = 0; i < p.n; i++) {
            if (p.field == 2) {
                witness[i] = (uint8_t)bit(c.x, i);
                witness[p.n + i] = (uint8_t)bit(c.z, i);
            } else {
                witness[i] = (uint8_t)proj(c, i);
            }
        }
    }
    if (coeffs) {
        memset(coeffs, 0, (size_t)p.K_in);
        for (int i = 0; i < p.k_eff; i++)
            coeffs[p.kept[i]] = (uint8_t)(bit(k.p[0], i) | (bit(k.p[1], i) << 1));
    }
    return P_OK;
}

int plan_decode(const Plan& p, const WitnessSlot& s, uint8_t* witness, uint8_t* coeffs) {
    if (s.gamma == DIST_SEED_GAMMA) {  // the planner's seed codeword
        if ((int)s.weight != vec_weight(p.seed_vec, p.W)) return P_EINVAL;
        return plan_decode_coef(p, p.seed_coef, (int)s.weight, witness, coeffs, &p.seed_vec);
    }
    if (s.gamma >= p.gammas.size() || s.count == 0 || s.count > DIST_MAXR) return P_EINVAL;
    const Gamma& G = p.gammas[s.gamma];
    Vec c;
    Coef k;
    memset(&c, 0, sizeof c);
    memset(&k, 0, sizeof k);
    for (uint32_t t = 0; t < s.count; t++) {
        int u = s.unit[t], e = s.digit[t];
        const Unit* x = u < (int)G.A.size() ? &G.A[u]
                        : (u - (int)G.A.size() < (int)G.B.size() ? &G.B[u - G.A.size()] : nullptr);
        if (!x || e >= x->nrep) return P_EINVAL;
        vxor(c, x->rep[e]);
        cxor(k, x->coef[e]);
    }
    if ((int)s.weight != vec_weight(c, p.W)) return P_EINVAL;
    // the coefficients must rebuild the same codeword from the input rows
    return plan_decode_coef(p, k, (int)s.weight, witness, coeffs, &c);
}

}  // namespace dist
