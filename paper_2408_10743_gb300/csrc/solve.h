// solve.h -- the round loop of Brouwer-Zimmermann (steps S3 and S6), generic
// over the executor that runs one enumeration step.
//
// Bounds (Section 2.1; Section 2.3 for the package argument and the bound of
// the second matrix): a combination that uses g units of a matrix weighs at
// least g - f on that matrix's pivot qubits (f = its free rows), and the
// matrices' pivot sets are disjoint.  Once round r of J[0..jpos] and round r-1
// of the others are finished, every codeword not yet seen has at least r+1
// (resp. r) units in each matrix, so it weighs at least
//     L = sum_{t <= jpos} max(0, r + 1 - f_t) + sum_{t > jpos} max(0, r - f_t).
// The upper bound U is the lightest codeword found.  Stop when L >= U; the
// kernels also stop early as soon as U <= the L already established.
#pragma once
#include <string.h>
#include <time.h>

#include <algorithm>

#include "../../include/dist.h"
#include "plan.h"

namespace dist {

struct StepResult {
    uint32_t U;
    uint32_t status;
    unsigned long long codewords;  // cumulative over the solve
};

static inline double wall_now() {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

// Exec must provide:
//   int reset();                                   // U = DIST_WINF, counters and slots cleared
//   int run(EnumParams& ep, double deadline_wall, StepResult* out);
//   int read_slot(uint32_t w, WitnessSlot* out);
//   int target_warps() const;
//   double gpu_seconds() const; unsigned long long launches() const;
template <class Exec>
int solve_loop(const Plan& p, Exec& ex, double time_limit_s, dist_result* out) {
    const double t0 = wall_now();
    const double deadline = time_limit_s > 0 ? t0 + time_limit_s : 0.0;
    memset(out, 0, sizeof *out);
    out->k_eff = p.k_eff;
    out->n_gamma = (int)p.J.size();
    int rc = ex.reset();
    if (rc) return rc;
    int L = plan_initial_bound(p);
    uint32_t U = DIST_WINF;
    StepResult sr{DIST_WINF, 0, 0};
    int status = DIST_OK;
    bool done = false;
    for (int r = 1; !done; r++) {
        for (int jpos = 0; jpos < (int)p.J.size() && !done; jpos++) {
            EnumParams ep;
            unsigned long long cw = 0;
            int prc = plan_step(p, jpos, r, L, ex.target_warps(), &ep, &cw);
            if (prc) {
                status = prc == P_ERANGE ? DIST_ERANGE : DIST_EINVAL;
                done = true;
                break;
            }
            out->rounds = r;
            rc = ex.run(ep, deadline, &sr);
            if (rc) return rc;
            U = sr.U;
            if (U != DIST_WINF && (int)U <= L) {  // certified by a bound already in force
                done = true;
                break;
            }
            if (sr.status & 2u) {                  // the kernel hit the deadline
                status = DIST_EINCOMPLETE;
                done = true;
                break;
            }
            L = plan_lower_bound(p, r, jpos);
            if (L == (int)DIST_WINF) {             // a matrix has been enumerated completely
                done = true;
                break;
            }
            if (U != DIST_WINF && L >= (int)U) {
                done = true;
                break;
            }
            if (deadline > 0 && wall_now() > deadline) {
                status = DIST_EINCOMPLETE;
                done = true;
                break;
            }
        }
    }
    out->codewords = sr.codewords;
    out->gpu_seconds = ex.gpu_seconds();
    out->launches = ex.launches();
    if (U == DIST_WINF) {
        out->status = status != DIST_OK ? status : DIST_EZERO;
        out->seconds = wall_now() - t0;
        return out->status;
    }
    out->d = (int)U;
    out->lower = (status == DIST_OK) ? (int)U : std::min(L, (int)U);
    WitnessSlot s;
    rc = ex.read_slot(U, &s);
    if (rc) return rc;
    if (s.claim == 0 || plan_decode(p, s, out->witness, out->coeffs) != P_OK) {
        out->status = DIST_EINTERNAL;
        out->seconds = wall_now() - t0;
        return DIST_EINTERNAL;
    }
    out->status = status;
    out->seconds = wall_now() - t0;
    return status;
}

}  // namespace dist
