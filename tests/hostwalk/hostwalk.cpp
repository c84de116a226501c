// hostwalk.cpp -- TEST HARNESS ONLY.  Runs the library's planner, round loop
// and the exact lane code of the enumeration kernel (walk.cuh) on the CPU,
// one simulated lane after another, so that tests can check the enumeration
// logic against the oracle without a GPU.  Not part of libdist.
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "plan.h"
#include "solve.h"
#include "walk.cuh"

using namespace dist;

namespace {

struct HostSink {
    Scratch* scr;
    bool poll(uint32_t& thr, int L_before) {
        uint32_t u = scr->U;
        if (u < thr) thr = u;
        return (int)u <= L_before;
    }
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
            for (int t = 0; t < g.a * 3; t++) {
                r0[t].x = src[(t * 2 + 0) * ep.W];
                r0[t].z = src[(t * 2 + 1) * ep.W];
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
            int sgi = 0;
            while (sgi + 1 < (int)lp.segs.size() && lp.segs[sgi + 1].chunk_base <= chunk) ++sgi;
            const SegDesc& sg = lp.segs[sgi];
            if ((int)scr.U <= sg.L_before) break;
            const GammaDesc& g = lp.g[sg.g];
            LaneCtx C;
            C.reps = sm.data() + g.s_rep;
            C.r0 = reinterpret_cast<const U2*>(sm.data() + g.s_r0);
            C.flags = sm.data() + g.s_flag;
            C.coefs = p->tables.data() + g.coef_off;
            C.binom = sbin;
            C.bstride = lp.bcols;
            C.outside = ep.outside;
            C.a = g.a; C.b = g.b; C.W = ep.W; C.CW = ep.CW; C.r = sg.r;
            C.gamma = g.gamma; C.proj = ep.proj; C.exclude = ep.exclude;
            C.L_before = sg.L_before;
            unsigned long long total = sg.NA * sg.NB;
            for (int lane = 0; lane < 32; lane++) {
                unsigned long long lo = (chunk - sg.chunk_base) * 32ull * sg.spl + (unsigned long long)lane * sg.spl;
                if (lo >= total) continue;
                unsigned long long hi = lo + sg.spl < total ? lo + sg.spl : total;
                uint32_t thr = DIST_WINF;
                scr.codewords += walk_range(C, sink, thr, sg, lo, hi);
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
