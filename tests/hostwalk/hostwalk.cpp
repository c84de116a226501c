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
    int L_prev;
    bool poll(uint32_t& thr) {
        uint32_t u = scr->U;
        if (u < thr) thr = u;
        return (int)u <= L_prev;
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
    int target_warps() const { return warps; }
    double gpu_seconds() const { return 0.0; }
    unsigned long long launches() const { return nlaunch; }
    int run(EnumParams& ep, double, StepResult* out) {
        const Gamma& G = p->gammas[ep.gamma];
        std::vector<U2> r0((size_t)ep.a * 3);
        for (int t = 0; t < ep.a * 3; t++) {
            r0[t].x = G.dev_reps[((size_t)t * 2 + 0) * ep.W];
            r0[t].z = G.dev_reps[((size_t)t * 2 + 1) * ep.W];
        }
        LaneCtx C;
        C.reps = G.dev_reps.data();
        C.r0 = r0.data();
        C.coefs = G.dev_coefs.data();
        C.binom = binom.data();
        C.outside = ep.outside;
        C.a = ep.a; C.b = ep.b; C.W = ep.W; C.CW = ep.CW; C.r = ep.r;
        C.gamma = ep.gamma; C.proj = ep.proj; C.exclude = ep.exclude;
        HostSink sink{&scr, ep.L_prev};
        nlaunch++;
        for (unsigned long long chunk = 0; chunk < ep.nchunks; chunk++) {
            int sgi = 0;
            while (sgi + 1 < ep.nseg && ep.seg[sgi + 1].chunk_base <= chunk) ++sgi;
            const SegDesc& sg = ep.seg[sgi];
            unsigned long long total = sg.NA * sg.NB;
            for (int lane = 0; lane < 32; lane++) {
                unsigned long long lo = (chunk - sg.chunk_base) * 32ull * sg.spl + (unsigned long long)lane * sg.spl;
                if (lo >= total) continue;
                unsigned long long hi = lo + sg.spl < total ? lo + sg.spl : total;
                uint32_t thr = DIST_WINF;
                scr.codewords += walk_range(C, sink, thr, sg, lo, hi);
            }
            if ((int)scr.U <= ep.L_prev) break;
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
    rd_unrank(B.data(), rank0, t, s);
    for (int c = 0; c < count; c++) {
        memcpy(out + (size_t)c * t, s, (size_t)t);
        if (c + 1 < count) rd_next(s, t, n);
    }
}
