// solve.h -- the round loop of Brouwer-Zimmermann (steps S3 and S6), generic
// over the executor that runs one launch of enumeration steps.
//
// Bounds (Section 2.1; Section 2.3 for the package argument and the bound of
// the second matrix): a combination that uses g units of a matrix weighs at
// least g - f on that matrix's pivot qubits (f = its free rows), and the
// matrices' pivot sets are disjoint.  Once round r of J[0..jpos] and round r-1
// of the others are finished, every codeword not yet seen has at least r+1
// (resp. r) units in each matrix, so it weighs at least
//     L = sum_{t <= jpos} max(0, r + 1 - f_t) + sum_{t > jpos} max(0, r - f_t).
// The upper bound U is the lightest codeword found.
//
// One launch runs a run of consecutive steps; each segment carries L_before,
// the bound that holds once every earlier step is complete, and the kernel
// drops work of a segment as soon as U <= its L_before.  After the launch let
// s be the first step with U <= L_before(s).  No chunk of a step before s was
// dropped (a drop needs U <= L_before there, and U only decreases), so all
// steps before s are complete, every unseen codeword weighs at least
// L_before(s) >= U, and d = U.  If no such s exists nothing was dropped and
// the bound after the launch's last step holds; d = U once it reaches U.
// A launch that ends on its time budget drops claimed chunks of any step, so
// the argument does not apply to it: after such a launch only the bound
// before its first step holds.
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

// Work allowed in one launch (codewords, ~ a few seconds of a GB300).
static const double kLaunchCodewords = 2e13;

// The bound a solve starts from: the lightest representative (outside S in
// exclusion mode), DIST_WINF if there is none.
static inline int seed_bound(const Plan& p) { return p.n_stab > 0 ? p.u0_excl : p.u0; }
static inline const WitnessSlot& seed_slot(const Plan& p) { return p.n_stab > 0 ? p.u0_excl_slot : p.u0_slot; }

// Exec must provide:
//   int reset();                                   // U = DIST_WINF, counters and slots cleared
//   int seed(uint32_t U0, const WitnessSlot& s);   // U = U0 with s in slot[U0]
//   int run(const LaunchPlan& lp, double deadline_wall, StepResult* out);
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
    int r = 1, jpos = 0;
    // The lightest representative is a codeword (outside S in exclusion
    // mode): start from it, so that no lane ever filters against "infinity".
    const int ubound0 = seed_bound(p);
    if (ubound0 < (int)DIST_WINF) {
        rc = ex.seed((uint32_t)ubound0, seed_slot(p));
        if (rc) return rc;
        U = (uint32_t)ubound0;
        sr.U = U;
    }
    for (;;) {
        LaunchPlan lp;
        const int ub = std::min<int>((int)U, ubound0);
        int prc = plan_launch(p, r, jpos, L, ub, ex.target_warps(), kLaunchCodewords, &lp);
        if (prc) {
            status = prc == P_ERANGE ? DIST_ERANGE : DIST_EINVAL;
            break;
        }
        rc = ex.run(lp, deadline, &sr);
        if (rc) return rc;
        U = sr.U;
        if (sr.status & 2u) {
            // The kernel spent its time budget and dropped the chunks it had
            // not run, in any step of the launch: only the bound that held
            // before the launch is known to hold after it.
            L = lp.step_L_before[0];
            if (U == DIST_WINF || (int)U > L) status = DIST_EINCOMPLETE;
            break;
        }
        bool certified = false;
        for (size_t s = 0; s < lp.step_r.size(); s++) {
            if (U != DIST_WINF && (int)U <= lp.step_L_before[s]) {
                certified = true;
                L = lp.step_L_before[s];
                break;
            }
            out->rounds = lp.step_r[s];  // last step known to be complete so far
        }
        if (certified) break;
        L = plan_lower_bound(p, lp.step_r.back(), lp.step_jpos.back());
        if (L == (int)DIST_WINF) break;  // a matrix has been enumerated completely
        if (U != DIST_WINF && L >= (int)U) break;
        r = lp.next_r;
        jpos = lp.next_jpos;
        if (deadline > 0 && wall_now() > deadline) {
            status = DIST_EINCOMPLETE;
            break;
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
