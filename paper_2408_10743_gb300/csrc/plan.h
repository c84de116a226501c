// plan.h -- host side of the distance computation (no CUDA calls):
//   S1 ingest + rank reduction, S2 package diagonalization into generator
//   matrices Gamma_1..Gamma_m on disjoint qubit sets, S3 the lower-bound
//   schedule, the per-launch work description, and S6 witness decoding.
#pragma once
#include <stdint.h>

#include <vector>

#include "dist_types.h"

namespace dist {

// A vector of F2^{2n} as two bit-planes; for F4 inputs the same planes hold
// a + alpha b (x = coefficient of 1, z = coefficient of alpha).
struct Vec {
    uint32_t x[DIST_MAXW];
    uint32_t z[DIST_MAXW];
};

// Coefficient vector over the kept basis rows.  F2: plane 0 holds one bit per
// row.  F4: planes 0/1 hold the F4 scalar a + alpha b of each row.
struct Coef {
    uint32_t p[2][DIST_MAXCW];
};

enum UnitKind { UNIT_PACKAGE2 = 0, UNIT_PACKAGE1 = 1, UNIT_FREE = 2 };

// One element of an enumeration: a package of rows sharing a pivot qubit, or a
// free row.  A-units carry three representatives with rep[0]^rep[1]^rep[2]=0
// (rank-2 package {g, h, g+h}, or an F4 row {g, alpha g, alpha^2 g});
// B-units carry one.
struct Unit {
    int kind;
    int qubit;   // pivot qubit, -1 for a free row
    int nrep;    // 1 or 3
    Vec rep[3];  // original qubit order
    Coef coef[3];
};

struct Gamma {
    std::vector<Unit> A, B;
    int f = 0;                    // free rows (no pivot qubit)
    int npack = 0;                // units with a pivot qubit
    std::vector<int> pivots;      // pivot qubits, in pivot order
    std::vector<int> perm;        // device position p -> original qubit
    std::vector<uint32_t> dev_reps;   // [u][3][2][W], device qubit order
    std::vector<uint32_t> dev_coefs;  // [u][3][2][CW]
    uint32_t a_all = 0;                 // AND of the A-units' flags
    std::vector<uint32_t> dev_flags;  // [u]: bit 0 package with pivot outside word 0, bit 1 outside words 0-1
    std::vector<uint32_t> dev_r0;     // [a][3][2]: word 0 of the A-units' representatives
    std::vector<uint32_t> dev_r1;     // [a][3][2]: word 1 (zeros if W = 1)
    int t1 = 0;                       // filter switch level (see walk.cuh)
    uint32_t rep_off = 0, coef_off = 0, flag_off = 0, r0_off = 0, r1_off = 0;  // offsets in Plan::tables
    bool tables_built = false;        // dev_* and perm filled
    int units() const { return (int)(A.size() + B.size()); }
};

struct Plan {
    int n = 0, field = 2, W = 1, CW = 1;
    int K_in = 0;                 // input rows
    int k_eff = 0;                // rank: F2 rows (field 2) or F4 rows (field 4)
    std::vector<Vec> input;       // input rows as planes
    std::vector<int> kept;        // input row index of every basis row
    std::vector<Vec> basis;
    int n_stab = 0, s_rank = 0;   // exclusion: S = span(first n_stab input rows)
    uint32_t outside[DIST_MAXCW] = {0};
    std::vector<Gamma> gammas;    // every matrix built
    std::vector<int> J;           // matrices enumerated, in order
    std::vector<uint32_t> tables; // every matrix's device tables, concatenated
    int u0 = 0;                   // smallest weight among all representatives
    int u0_excl = 0;              // same, among representatives outside S (exclusion)
    WitnessSlot u0_slot{}, u0_excl_slot{};  // which representative reaches them
    Vec seed_vec{};               // a slot with gamma DIST_SEED_GAMMA names this codeword
    Coef seed_coef{};
    int d_est = 0;                // random-code estimate used to choose J
};

// Consecutive enumeration steps (round r of matrix J[jpos]) run by one launch.
struct LaunchPlan {
    std::vector<SegDesc> segs;
    std::vector<GammaDesc> g;
    std::vector<int> step_r, step_jpos, step_L_before;
    std::vector<int> step_seg0;                     // first segment of each step
    std::vector<unsigned long long> step_chunk0;    // first chunk of each step (nchunks if none)
    int W = 1, CW = 1, proj = 0, exclude = 0;
    int brows = 0, bcols = 0;
    uint32_t s_binom = 0, s_segs = 0, s_words = 0;  // shared-memory layout
    unsigned long long nchunks = 0;
    double codewords = 0;         // if every step completes
    int next_r = 0, next_jpos = 0;
    std::vector<SegDesc> raw_segs;  // one segment per (step, i) before chunking
    std::vector<int> raw_step_seg0;
};

enum { P_OK = 0, P_EINVAL = -1, P_ENOMEM = -2, P_EZERO = -6, P_ERANGE = -9 };

// Chunk granularity used by plan_launch (process-wide, set by the tuner):
// each step of a launch is cut into about chunks_per_warp warp-chunks per
// resident warp, and a lane chunk holds at most 2^lane_cap_log2 and at least
// 2^lane_floor_log2 codewords.
struct Tuning {
    int chunks_per_warp = 6;
    int lane_cap_log2 = 14;
    int lane_floor_log2 = 12;
};
Tuning tuning_get();

// Qubit orders plan_build tries for a code whose estimated work exceeds
// 5e8 codewords and whose matrices in J have free rows (0 = index order
// only; default 8, range 0..256; process-wide).
int plan_search_trials();
void plan_set_search_trials(int t);
// Largest number of generator matrices the choice of J may take (0: no
// limit beyond the policy's own choice).
int plan_gamma_limit();
void plan_set_gamma_limit(int m);
void tuning_set(const Tuning& t);

// S1 + S2 + choice of J.  gen layout: field 2 -> K x 2n bytes {0,1} (x | z);
// field 4 -> K x n bytes {0..3}, v = a + 2b for a + alpha b.
int plan_build(const uint8_t* gen, int n, int K, int field, Plan* p);

// Minimum over C minus span(first n_stab input rows); 0 switches it off.
int plan_set_exclude(Plan* p, int n_stab);

// Lower bound on every codeword not yet enumerated once J[0..jpos] have
// finished round r and J[jpos+1..] round r-1.  Returns DIST_WINF when some
// matrix has enumerated all of its combinations (nothing left unseen).
int plan_lower_bound(const Plan& p, int r, int jpos);
int plan_initial_bound(const Plan& p);

// Codewords (subset x representative choices) of round r of matrix g.
double plan_round_count(const Plan& p, int g, int r);

// Steps from (r, jpos) onward for one launch: at least one, then more while
// the estimated work stays under max_codewords, the segment table fits, and
// the bound in force before the next step is still below U_bound (a step
// with L_before >= U can never be needed).  L_prev is the bound in force
// before (r, jpos).  Returns P_ERANGE if r exceeds the device walk's limits.
int plan_launch(const Plan& p, int r, int jpos, int L_prev, int U_bound, int target_warps,
                double max_codewords, LaunchPlan* lp);
// Re-cuts a planned launch into chunks for another resident-warp count (the
// batch engine gives each code of a slice its share of the warps).
int plan_rechunk(LaunchPlan* lp, int target_warps);

// What a code's state means after a launch that may have stopped early
// (time budget).  next = chunks claimed so far (all claimed chunks finished).
// CERTIFIED: d = U (or no codeword if U = DIST_WINF).  CONTINUE: resume the
// same plan.  REPLAN: every planned step finished below U; plan from
// (lp.next_r, lp.next_jpos) with the bound L_after.
enum { SLICE_CONTINUE = 0, SLICE_CERTIFIED = 1, SLICE_REPLAN = 2 };
struct SliceVerdict {
    int kind;
    int L;           // certifying bound (CERTIFIED) or bound in force for the next plan (REPLAN)
    int last_round;  // last round known complete
};
SliceVerdict plan_after_slice(const Plan& p, const LaunchPlan& lp, uint32_t U, unsigned long long next);

// Lower bound established by a partly run plan: the L_before of its first
// step that is not complete (or the bound after its last step).
int plan_partial_bound(const Plan& p, const LaunchPlan& lp, unsigned long long next);

// Fills the launch-independent part of EnumParams (pointers stay null).
void plan_params(const Plan& p, const LaunchPlan& lp, EnumParams* ep);

// Rebuilds the codeword recorded in a witness slot.  witness: 2n bytes (F2)
// or n bytes (F4); coeffs: K_in bytes over the input rows (F2 bits or F4
// symbols).  Checks the weight and that the coefficients reproduce it.
int plan_decode(const Plan& p, const WitnessSlot& s, uint8_t* witness, uint8_t* coeffs);
// The codeword with coefficients k over the basis: checks that it lies
// outside S (exclusion), has symplectic weight `weight` and (if given) equals
// *expect, then writes it and its coefficients over the input rows as
// plan_decode does.
int plan_decode_coef(const Plan& p, const Coef& k, int weight, uint8_t* witness, uint8_t* coeffs,
                     const Vec* expect = nullptr);

// Stabilizer-code front end (stab.cpp): from m generator rows (x | z) of the
// classical stabilizer code S of an [[n, k]] qubit code, a generator matrix
// of its normalizer N = S^{perp_s} whose first *n_stab rows are a basis of S
// (K = n + k rows, n_stab = n - k); for k = 0 a basis of S with n_stab = 0.
// P_EINVAL for bad input or generators that do not commute, P_EZERO if S = 0.
int stab_normalizer(const uint8_t* stab, int n, int m, std::vector<uint8_t>* gen, int* K, int* n_stab);

// Saturating binomial table [(DIST_MAXU+1) x (DIST_MAXR+1)].
void binom_table(unsigned long long* tab);

int vec_weight(const Vec& v, int W);

}  // namespace dist
