// hostwalk.cpp -- TEST HARNESS ONLY.  Runs the library's planner, round loop
// and the exact lane code of the enumeration kernel (walk.cuh) on the CPU,
// one simulated lane after another, so that tests can check the enumeration
// logic against the oracle without a GPU.  Not part of libdist.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "plan.h"
#include "solve.h"
#include "isosplit.cuh"
#include "rdorder.cuh"
#include "walk.cuh"

using namespace dist;

namespace {

struct HostSink {
    Scratch* scr;
    bool vote_any(bool p) { return p; }
    uint32_t peek() { return scr->U; }
    void record(uint32_t w, int gamma, int count, const uint8_t* units, const uint8_t* digits) {
        if (w < scr->U) scr->U = w;
        WitnessSlot* s = &scr->slot[w];
        if (s->claim == 0) {
            s->claim = 1;
            s->gamma = (uint32_t)gamma;
            s->count = (uint32_t)count;
            s->weight = w;
            for (int k = 0; k < count; k++) {
                s->unit[k] = units[k];
                s->digit[k] = digits[k];
            }
        }
    }
};

// Runs a launch plan chunk by chunk, lane by lane, exactly as the kernel
// would, but sequentially.
struct HostExec {
    const Plan* p;
    Scratch scr;
    std::vector<unsigned long long> binom;
    int warps = 4;
    unsigned long long nlaunch = 0;
    // > 0: a launch stops after this many chunks as if its time budget ran
    // out (status bit 1, the rest of its chunks dropped), like the kernel's
    // budget stop
    long long stop_after = 0;
    HostExec(const Plan* pp) : p(pp), binom((DIST_MAXU + 1) * (DIST_MAXR + 1)) {
        binom_table(binom.data());
    }
    int reset() {
        memset(&scr, 0, sizeof scr);
        scr.U = DIST_WINF;
        return 0;
    }
    int seed(uint32_t U0, const WitnessSlot& s) {
        scr.U = U0;
        scr.slot[U0] = s;
        return 0;
    }
    int target_warps() const { return warps; }
    double gpu_seconds() const { return 0.0; }
    unsigned long long launches() const { return nlaunch; }
    int run(const LaunchPlan& lp, double, StepResult* out) {
        EnumParams ep;
        plan_params(*p, lp, &ep);
        // the shared-memory image the kernel would build
        std::vector<uint32_t> sm(lp.s_words + 2, 0);
        for (const GammaDesc& g : lp.g) {
            const uint32_t* src = p->tables.data() + g.rep_off;
            for (int t = 0; t < (g.a + g.b) * 6 * ep.W; t++) sm[g.s_rep + t] = src[t];
            U2* r0 = reinterpret_cast<U2*>(sm.data() + g.s_r0);
            U2* r1 = reinterpret_cast<U2*>(sm.data() + g.s_r1);
            for (int t = 0; t < g.a * 3; t++) {
                r0[t].x = src[(t * 2 + 0) * ep.W];
                r0[t].z = src[(t * 2 + 1) * ep.W];
                r1[t].x = ep.W >= 2 ? src[(t * 2 + 0) * ep.W + 1] : 0u;
                r1[t].z = ep.W >= 2 ? src[(t * 2 + 1) * ep.W + 1] : 0u;
            }
            for (int t = 0; t < g.a + g.b; t++) sm[g.s_flag + t] = p->tables[g.flag_off + t];
        }
        unsigned long long* sbin = reinterpret_cast<unsigned long long*>(sm.data() + lp.s_binom);
        for (int t = 0; t < lp.brows * lp.bcols; t++) {
            int n = t / lp.bcols, k = t - n * lp.bcols;
            sbin[t] = binom[n * (DIST_MAXR + 1) + k];
        }
        HostSink sink{&scr};
        nlaunch++;
        for (unsigned long long chunk = 0; chunk < lp.nchunks; chunk++) {
            if (stop_after > 0 && chunk == (unsigned long long)stop_after) {
                scr.status |= 2u;
                break;
            }
            int sgi = 0;
            while (sgi + 1 < (int)lp.segs.size() && lp.segs[sgi + 1].chunk_base <= chunk) ++sgi;
            const SegDesc& sg = lp.segs[sgi];
            if ((int)scr.U <= sg.L_before) break;
            const GammaDesc& g = lp.g[sg.g];
            LaneCtx C;
            C.reps = sm.data() + g.s_rep;
            C.r0 = reinterpret_cast<const U2*>(sm.data() + g.s_r0);
            C.r1 = reinterpret_cast<const U2*>(sm.data() + g.s_r1);
            C.flags = sm.data() + g.s_flag;
            C.t1 = g.t1;
            C.a_all = g.a_all;
            C.coefs = p->tables.data() + g.coef_off;
            C.binom = sbin;
            C.bstride = lp.bcols;
            C.outside = ep.outside;
            C.a = g.a; C.b = g.b; C.W = ep.W; C.CW = ep.CW;
            C.gamma = g.gamma; C.proj = ep.proj; C.exclude = ep.exclude;
            for (int lane = 0; lane < 32; lane++) {
                unsigned long long lo, hi;
                if (!seg_lane_range(sg, chunk, lane, lo, hi)) continue;
                uint32_t thr = DIST_WINF;
                scr.codewords += walk_range(C, sink, thr, sg, lo, hi, sink.peek());
            }
        }
        out->U = scr.U;
        out->status = scr.status;
        out->codewords = scr.codewords;
        return 0;
    }
    int read_slot(uint32_t w, WitnessSlot* s) {
        *s = scr.slot[w];
        return 0;
    }
};

}  // namespace


// 64-bit FNV-1a digest of what the first enumeration launch of a solve
// reads: ties a committed ncu capture of that launch to the planner's
// current output (tests compare it with the digest recorded beside the
// capture).
namespace {
// reads on a device with target_warps resident warps, under the current
// tuning: the device tables, the seed bound and its witness slot, the launch
// parameters (device pointers and time budget excluded) and the segment
// table.  Equal digests hand the kernel byte-identical work, so a profile of
// that launch stays valid while the kernel's own sources are unchanged.
unsigned long long first_launch_digest(const Plan& p, int target_warps) {
    unsigned long long h = 1469598103934665603ull;
    auto put = [&h](const void* d, size_t n) {
        const unsigned char* c = static_cast<const unsigned char*>(d);
        for (size_t i = 0; i < n; i++) {
            h ^= c[i];
            h *= 1099511628211ull;
        }
    };
    const int ub = seed_bound(p);
    put(&target_warps, sizeof target_warps);
    put(p.tables.data(), p.tables.size() * sizeof(uint32_t));
    put(&ub, sizeof ub);
    if (ub < (int)DIST_WINF) put(&seed_slot(p), sizeof(WitnessSlot));
    // solve_loop's first step: round 1 of J[0], from the initial bound
    LaunchPlan lp;
    const int rc = plan_launch(p, 1, 0, plan_initial_bound(p), ub, target_warps, kLaunchCodewords, &lp);
    put(&rc, sizeof rc);
    if (rc == P_OK) {
        EnumParams ep;
        plan_params(p, lp, &ep);  // zeroes the pointers and the budget
        ep.first_static = (uint32_t)ub <= (uint32_t)p.d_est ? 1 : 0;
        ep.two_word = enum_two_word(ep, (uint32_t)ub);
        put(&ep, sizeof ep);
        put(lp.segs.data(), lp.segs.size() * sizeof(SegDesc));
    }
    return h;
}

}  // namespace

extern "C" int hw_launch_digest(const uint8_t* gen, int n, int K, int field, int n_stab, int target_warps,
                                unsigned long long* digest) {
    Plan p;
    int rc = plan_build(gen, n, K, field, &p);
    if (rc) return rc;
    if (n_stab) {
        rc = plan_set_exclude(&p, n_stab);
        if (rc) return rc;
    }
    *digest = first_launch_digest(p, target_warps);
    return 0;
}

extern "C" void hw_set_tuning(int chunks_per_warp, int lane_cap_log2, int lane_floor_log2) {
    Tuning t = tuning_get();
    t.chunks_per_warp = chunks_per_warp;
    t.lane_cap_log2 = lane_cap_log2;
    t.lane_floor_log2 = lane_floor_log2;
    tuning_set(t);
}

extern "C" int hw_solve(const uint8_t* gen, int n, int K, int field, int n_stab, int warps,
                        dist_result* out) {
    Plan p;
    int rc = plan_build(gen, n, K, field, &p);
    if (rc) return rc;
    if (n_stab) {
        rc = plan_set_exclude(&p, n_stab);
        if (rc) return rc;
    }
    HostExec ex(&p);
    ex.warps = warps;
    return solve_loop(p, ex, 0.0, out);
}

// solve_loop with launches that stop after stop_after chunks as the kernel
// does when its time budget runs out.
extern "C" int hw_solve_stop(const uint8_t* gen, int n, int K, int field, int warps, long long stop_after,
                             dist_result* out) {
    Plan p;
    int rc = plan_build(gen, n, K, field, &p);
    if (rc) return rc;
    HostExec ex(&p);
    ex.warps = warps;
    ex.stop_after = stop_after;
    return solve_loop(p, ex, 0.0, out);
}

// The batch engine's per-code life cycle on the CPU: the whole remaining plan
// in one launch plan, executed in slices that stop after a random number of
// chunks (a time budget), with the kernel's skip rule, until the after-slice
// verdict certifies d.  Exercises resumption and re-planning.
extern "C" int hw_solve_sliced(const uint8_t* gen, int n, int K, int field, int n_stab,
                               unsigned seed, int max_seg_per_plan, dist_result* out) {
    Plan p;
    int rc = plan_build(gen, n, K, field, &p);
    if (rc) return rc;
    if (n_stab) {
        rc = plan_set_exclude(&p, n_stab);
        if (rc) return rc;
    }
    memset(out, 0, sizeof *out);
    HostExec ex(&p);
    ex.warps = 3;
    ex.reset();
    const int u0 = p.n_stab > 0 ? p.u0_excl : p.u0;
    if (u0 < (int)DIST_WINF) ex.seed((uint32_t)u0, p.n_stab > 0 ? p.u0_excl_slot : p.u0_slot);
    int L = plan_initial_bound(p), r = 1, jpos = 0;
    unsigned lcg = seed * 2654435761u + 12345u;
    for (int plans = 0; plans < 1000; plans++) {
        LaunchPlan lp;
        rc = plan_launch(p, r, jpos, L, u0, ex.warps, max_seg_per_plan > 0 ? 1.0 : 1e300, &lp);
        if (rc) return rc;
        if (max_seg_per_plan > 0 && (int)lp.step_r.size() > 1) {
            // force short plans (one step) to exercise re-planning
            lp = LaunchPlan();
            rc = plan_launch(p, r, jpos, L, u0, ex.warps, 0.0, &lp);
            if (rc) return rc;
        }
        std::vector<uint32_t> flags;
        unsigned long long next = 0;
        for (;;) {
            lcg = lcg * 1664525u + 1013904223u;
            unsigned long long slice_chunks = 1 + (lcg >> 8) % 7;
            // run up to slice_chunks chunks of this plan from `next`, as a launch would
            LaunchPlan part = lp;
            EnumParams ep;
            plan_params(p, lp, &ep);
            std::vector<uint32_t> sm(lp.s_words + 2, 0);
            for (const GammaDesc& g : lp.g) {
                const uint32_t* src = p.tables.data() + g.rep_off;
                for (int t = 0; t < (g.a + g.b) * 6 * ep.W; t++) sm[g.s_rep + t] = src[t];
                U2* r0 = reinterpret_cast<U2*>(sm.data() + g.s_r0);
                U2* r1 = reinterpret_cast<U2*>(sm.data() + g.s_r1);
                for (int t = 0; t < g.a * 3; t++) {
                    r0[t].x = src[(t * 2 + 0) * ep.W];
                    r0[t].z = src[(t * 2 + 1) * ep.W];
                    r1[t].x = ep.W >= 2 ? src[(t * 2 + 0) * ep.W + 1] : 0u;
                    r1[t].z = ep.W >= 2 ? src[(t * 2 + 1) * ep.W + 1] : 0u;
                }
                for (int t = 0; t < g.a + g.b; t++) sm[g.s_flag + t] = p.tables[g.flag_off + t];
            }
            unsigned long long* sbin = reinterpret_cast<unsigned long long*>(sm.data() + lp.s_binom);
            for (int t = 0; t < lp.brows * lp.bcols; t++) {
                int nn = t / lp.bcols, k = t - nn * lp.bcols;
                sbin[t] = ex.binom[nn * (DIST_MAXR + 1) + k];
            }
            HostSink sink{&ex.scr};
            for (unsigned long long c = 0; c < slice_chunks && next < lp.nchunks; c++) {
                const unsigned long long chunk = next++;
                int sgi = 0;
                while (sgi + 1 < (int)lp.segs.size() && lp.segs[sgi + 1].chunk_base <= chunk) ++sgi;
                const SegDesc& sg = lp.segs[sgi];
                if ((int)ex.scr.U <= sg.L_before) {
                    next = lp.nchunks;  // the kernel's skip: the rest is not needed
                    break;
                }
                const GammaDesc& g = lp.g[sg.g];
                LaneCtx C;
                C.reps = sm.data() + g.s_rep;
                C.r0 = reinterpret_cast<const U2*>(sm.data() + g.s_r0);
                C.r1 = reinterpret_cast<const U2*>(sm.data() + g.s_r1);
                C.flags = sm.data() + g.s_flag;
                C.t1 = g.t1;
                C.a_all = g.a_all;
                C.coefs = p.tables.data() + g.coef_off;
                C.binom = sbin;
                C.bstride = lp.bcols;
                C.outside = ep.outside;
                C.a = g.a; C.b = g.b; C.W = ep.W; C.CW = ep.CW;
                C.gamma = g.gamma; C.proj = ep.proj; C.exclude = ep.exclude;
                for (int lane = 0; lane < 32; lane++) {
                    unsigned long long lo, hi;
                    if (!seg_lane_range(sg, chunk, lane, lo, hi)) continue;
                    uint32_t thr = DIST_WINF;
                    ex.scr.codewords += walk_range(C, sink, thr, sg, lo, hi, sink.peek());
                }
            }
            (void)part;
            const SliceVerdict v = plan_after_slice(p, lp, ex.scr.U, next);
            out->rounds = std::max(out->rounds, v.last_round);
            out->launches++;
            if (v.kind == SLICE_CERTIFIED) {
                out->codewords = ex.scr.codewords;
                out->k_eff = p.k_eff;
                if (ex.scr.U == DIST_WINF) return -6;
                out->d = (int)ex.scr.U;
                out->lower = out->d;
                WitnessSlot s = ex.scr.slot[ex.scr.U];
                if (s.claim == 0 || plan_decode(p, s, out->witness, out->coeffs) != P_OK) return -8;
                return 0;
            }
            if (v.kind == SLICE_REPLAN) {
                L = v.L;
                r = lp.next_r;
                jpos = lp.next_jpos;
                break;
            }
        }
    }
    return -8;
}

// The lower-bound schedule of the planner: out[r * nJ + jpos] = L after
// J[0..jpos] finish round r and the rest round r-1 (r = 0..rmax).
extern "C" int hw_plan_bounds(const uint8_t* gen, int n, int K, int field, int rmax, int* out,
                              int* J, int* nJ) {
    Plan p;
    int rc = plan_build(gen, n, K, field, &p);
    if (rc) return rc;
    *nJ = (int)p.J.size();
    for (int t = 0; t < *nJ; t++) J[t] = p.J[t];
    for (int r = 0; r <= rmax; r++)
        for (int t = 0; t < *nJ; t++) out[r * *nJ + t] = plan_lower_bound(p, r, t);
    return 0;
}

// Revolving-door helpers exactly as the kernel uses them.
extern "C" void hw_rd_walk(int n, int t, unsigned long long rank0, int count, uint8_t* out) {
    std::vector<unsigned long long> B((DIST_MAXU + 1) * (DIST_MAXR + 1));
    binom_table(B.data());
    uint8_t s[DIST_MAXR];
    rd_unrank(B.data(), DIST_MAXR + 1, n, rank0, t, s);
    for (int c = 0; c < count; c++) {
        memcpy(out + (size_t)c * t, s, (size_t)t);
        if (c + 1 < count) rd_next(s, t, n);
    }
}

// The first launch plan of a code at the given resident-warp count and chunk
// tuning, one row per segment: step, i, NA, NB, rank0, rank1, chunk_base, spl,
// codes.  Returns the number of rows (or a negative code); *nchunks gets the
// launch's chunk count.
extern "C" int hw_plan_segments(const uint8_t* gen, int n, int K, int field, int target_warps, int cpw,
                                int cap_log2, int floor_log2, unsigned long long* out, int max_rows,
                                unsigned long long* nchunks) {
    Plan p;
    int rc = plan_build(gen, n, K, field, &p);
    if (rc) return rc;
    const Tuning saved = tuning_get();
    Tuning t;
    t.chunks_per_warp = cpw;
    t.lane_cap_log2 = cap_log2;
    t.lane_floor_log2 = floor_log2;
    tuning_set(t);
    LaunchPlan lp;
    rc = plan_launch(p, 1, 0, plan_initial_bound(p), p.u0, target_warps, 2e13, &lp);
    tuning_set(saved);
    if (rc) return rc;
    if ((int)lp.segs.size() > max_rows) return -100;
    for (size_t k = 0; k < lp.segs.size(); k++) {
        int step = 0;
        while (step + 1 < (int)lp.step_seg0.size() && lp.step_seg0[step + 1] <= (int)k) ++step;
        const SegDesc& s = lp.segs[k];
        unsigned long long* row = out + k * 9;
        row[0] = (unsigned long long)step;
        row[1] = s.i;
        row[2] = s.NA;
        row[3] = s.NB;
        row[4] = s.rank0;
        row[5] = s.rank1;
        row[6] = s.chunk_base;
        row[7] = s.spl;
        row[8] = s.codes;
    }
    *nchunks = lp.nchunks;
    return (int)lp.segs.size();
}

// The steps of one launch planned from round 1 (bound U_bound, at most
// max_codewords): for step k, (r, jpos, L_before) in steps[3k..3k+2]; the
// L_before of every segment in seg_L.  Returns the number of steps (and
// *nseg), or a negative value on failure.
extern "C" int hw_plan_steps(const uint8_t* gen, int n, int K, int field, int U_bound, double max_codewords,
                             int* steps, int max_steps, int* seg_L, int max_segs, int* nseg) {
    Plan p;
    if (plan_build(gen, n, K, field, &p)) return -1;
    LaunchPlan lp;
    if (plan_launch(p, 1, 0, plan_initial_bound(p), U_bound, 2432, max_codewords, &lp)) return -2;
    const int ns = (int)lp.step_r.size();
    if (ns > max_steps || (int)lp.segs.size() > max_segs) return -3;
    for (int k = 0; k < ns; k++) {
        steps[3 * k] = lp.step_r[k];
        steps[3 * k + 1] = lp.step_jpos[k];
        steps[3 * k + 2] = lp.step_L_before[k];
    }
    for (size_t t = 0; t < lp.segs.size(); t++) seg_L[t] = lp.segs[t].L_before;
    *nseg = (int)lp.segs.size();
    return ns;
}

// Decodes a witness slot that names the plan's seed codeword (the path a
// codeword kept from another search trial takes): the seed is the sum of the
// given basis rows.  Returns its weight, or a negative value on failure.
extern "C" int hw_seed_decode(const uint8_t* gen, int n, int K, const int* rows, int nrows, uint8_t* witness,
                              uint8_t* coeffs) {
    Plan p;
    if (plan_build(gen, n, K, 2, &p)) return -1;
    Vec v;
    Coef k;
    memset(&v, 0, sizeof v);
    memset(&k, 0, sizeof k);
    for (int t = 0; t < nrows; t++) {
        const int i = rows[t];
        if (i < 0 || i >= p.k_eff) return -2;
        for (int w = 0; w < DIST_MAXW; w++) {
            v.x[w] ^= p.basis[i].x[w];
            v.z[w] ^= p.basis[i].z[w];
        }
        k.p[0][i >> 5] ^= 1u << (i & 31);
    }
    p.seed_vec = v;
    p.seed_coef = k;
    WitnessSlot s;
    memset(&s, 0, sizeof s);
    s.claim = 1;
    s.gamma = DIST_SEED_GAMMA;
    s.weight = (uint32_t)vec_weight(v, p.W);
    return plan_decode(p, s, witness, coeffs) == P_OK ? (int)s.weight : -3;
}

// 1 if planning for tw1 warps and re-cutting for tw2 gives the same launch as
// planning for tw2 directly, 0 if not, negative on a planning error.
extern "C" int hw_rechunk_same(const uint8_t* gen, int n, int K, int field, int tw1, int tw2) {
    Plan p;
    int rc = plan_build(gen, n, K, field, &p);
    if (rc) return rc;
    LaunchPlan a, b;
    if ((rc = plan_launch(p, 1, 0, plan_initial_bound(p), p.u0, tw1, 2e13, &a))) return rc;
    if ((rc = plan_launch(p, 1, 0, plan_initial_bound(p), p.u0, tw2, 2e13, &b))) return rc;
    plan_rechunk(&a, tw2);
    if (a.segs.size() != b.segs.size() || a.nchunks != b.nchunks || a.step_seg0 != b.step_seg0 ||
        a.step_chunk0 != b.step_chunk0 || a.s_words != b.s_words)
        return 0;
    return memcmp(a.segs.data(), b.segs.data(), a.segs.size() * sizeof(SegDesc)) == 0 ? 1 : 0;
}

// Walks count subsets of {0..n-1} in revolving-door order from rank rank0
// with rd_next_delta, recording each subset and the element that left and
// the one that entered at each step.
extern "C" void hw_rd_delta_walk(int n, int t, unsigned long long rank0, int count, uint8_t* out, int* moves) {
    std::vector<unsigned long long> B((DIST_MAXU + 1) * (DIST_MAXR + 1));
    binom_table(B.data());
    uint8_t s[DIST_MAXR];
    rd_unrank(B.data(), DIST_MAXR + 1, n, rank0, t, s);
    for (int k = 0; k < count; k++) {
        memcpy(out + (size_t)k * t, s, t);
        if (k + 1 < count) rd_next_delta(s, t, n, &moves[2 * k], &moves[2 * k + 1]);
    }
}

// Runs the split walk of the isometry kernel (isosplit.cuh) on the CPU for
// round r of K rows, unit by unit and thread by thread as the kernel does:
// each thread's lane-side sums stepped with split_next from one
// split_unrank, each tile entry by split_unrank.  Every (tile entry, lane
// value) pair is mapped back to its r-subset, whose colexicographic rank over
// all K rows is counted in hits[] (C(K, r) entries).  Also checks every sum
// the walk carries against the sum of the subset's rows (rows: K x 3 words,
// piv: K flags).  out[0] = units, out[1] = codewords counted per unit as the
// kernel counts them, out[2] = sums that differ, out[3] = lane values outside
// their thread's range.  Returns -1 if the split walk does not apply.
extern "C" int hw_split_cover(int K, int r, unsigned long long target, const uint32_t* rows, const uint8_t* piv,
                              uint32_t* hits, unsigned long long* out) {
    std::vector<unsigned long long> B((DIST_MAXU + 1) * (DIST_MAXR + 1));
    binom_table(B.data());
    SplitPlan sp;
    if (!split_plan(K, r, target, B.data(), &sp)) return -1;
    std::vector<SplitRow> srt(K), sdt(K);
    for (int t = 0; t < K; t++) srt[t] = SplitRow{rows[3 * t], rows[3 * t + 1], rows[3 * t + 2], piv[t]};
    for (int t = 0; t < K; t++) {
        const SplitRow a = srt[t], b = t + 1 < K ? srt[t + 1] : SplitRow{0u, 0u, 0u, 0u};
        sdt[t] = SplitRow{a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, b.np - a.np};
    }
    auto direct = [&](const uint8_t* s, int n) {
        SplitRow v{0u, 0u, 0u, 0u};
        for (int t = 0; t < n; t++) split_add(&v, srt[s[t]]);
        return v;
    };
    auto same = [](const SplitRow& a, const SplitRow& b) {
        return a.x == b.x && a.y == b.y && a.z == b.z && a.np == b.np;
    };
    unsigned long long counted = 0, bad = 0, outside = 0;
    for (unsigned long long u = 0; u < sp.units; u++) {
        const SplitUnit W = split_unit(sp.term, sp.nterms, u);
        const SplitTerm& S = sp.term[W.term];
        counted += (W.t_hi - W.t_lo) * (W.l_hi - W.l_lo);
        // tile entries of the unit
        std::vector<SplitRow> tile;
        std::vector<unsigned long long> trank;
        for (unsigned long long tr = W.t_lo; tr < W.t_hi; tr++) {
            SplitRow a;
            uint64_t TT;
            split_unrank(B.data(), srt.data(), S.tile_off, S.tile_kh, S.tile_t, tr, &TT, &a);
            uint8_t st[kSplitMaxT];
            split_rows(B.data(), S.tile_off, S.tile_kh, S.tile_t, tr, st);
            if (!same(direct(st, S.tile_t), a)) bad++;
            tile.push_back(a);
            trank.push_back(tr);
        }
        for (int tid = 0; tid < kSplitThreads; tid++) {
            unsigned long long q = W.l_lo + (unsigned long long)tid * W.per;
            const unsigned long long q_end = std::min(W.l_hi, q + W.per);
            uint64_t T = 0;
            SplitRow lv = {0u, 0u, 0u, 0u};
            if (q < q_end) split_unrank(B.data(), srt.data(), S.lane_off, S.lane_kh, S.lane_t, q, &T, &lv);
            for (uint32_t gi = 0; gi < S.groups; ++gi) {
                for (int j = 0; j < kSplitNB; j++) {
                    if (q >= q_end) break;
                    const unsigned long long lr = q;
                    if (lr < W.l_lo || lr >= W.l_hi) outside++;
                    uint8_t sl[kSplitMaxT];
                    split_rows(B.data(), S.lane_off, S.lane_kh, S.lane_t, lr, sl);
                    if (!same(direct(sl, S.lane_t), lv)) bad++;
                    for (size_t k = 0; k < tile.size(); k++) {
                        uint8_t s[2 * kSplitMaxT];
                        split_rows(B.data(), S.tile_off, S.tile_kh, S.tile_t, trank[k], s);
                        memcpy(s + S.tile_t, sl, S.lane_t);
                        std::sort(s, s + r);
                        unsigned long long rank = 0;
                        for (int t = 0; t < r; t++) rank += B[(size_t)s[t] * (DIST_MAXR + 1) + t + 1];
                        hits[rank]++;
                    }
                    ++q;
                    if (q < q_end) split_next(srt.data(), sdt.data(), S.lane_off, S.lane_t, &T, &lv);
                }
            }
        }
    }
    out[0] = sp.units;
    out[1] = counted;
    out[2] = bad;
    out[3] = outside;
    return 0;
}

// The split plan of round r of K rows for unit target `target` (isosplit.cuh):
// its terms (at most kSplitMaxTerms) and unit count.  Returns the number of
// terms, or -1 if the split walk does not apply.
extern "C" int hw_split_plan(int K, int r, unsigned long long target, SplitTerm* terms, unsigned long long* units) {
    std::vector<unsigned long long> B((DIST_MAXU + 1) * (DIST_MAXR + 1));
    binom_table(B.data());
    SplitPlan sp;
    if (!split_plan(K, r, target, B.data(), &sp)) return -1;
    for (int e = 0; e < sp.nterms; e++) terms[e] = sp.term[e];
    *units = sp.units;
    return sp.nterms;
}

extern "C" int hw_split_sizes(int* term_bytes, int* max_terms, int* threads, int* nb, int* tile) {
    *term_bytes = (int)sizeof(SplitTerm);
    *max_terms = kSplitMaxTerms;
    *threads = kSplitThreads;
    *nb = kSplitNB;
    *tile = kSplitTile;
    return 0;
}
