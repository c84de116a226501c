// dist_types.h -- limits and plain structs shared by the host planner, the
// enumeration kernel and the C-ABI layer of libdist.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define DIST_HD __host__ __device__ __forceinline__
#else
#define DIST_HD inline
#endif

#define DIST_MAXN 128          // qubits
#define DIST_MAXW 4            // 32-bit words per bit-plane (n <= 128)
#define DIST_MAXK 256          // F2 rows (F4 inputs: rows of the F2 view)
#define DIST_MAXCW 8           // 32-bit words of a coefficient plane (K <= 256)
#define DIST_MAXU 256          // enumeration units of one generator matrix
#define DIST_MAXR 32           // largest combination size walked on the device
#define DIST_MAXGAMMA 16
#define DIST_MAXSEG 256        // segments in one launch
#define DIST_WINF 0xFFFFu      // "no codeword yet" weight
#define DIST_FAST_MAX_DYN 20   // 3^20 < 2^32: the dynamic Gray counter fits in 32 bits
// Subsets of i A-units take the lane walk's fast path (a nine-entry register
// table, two register digits and a ternary Gray code over the rest) when
// they have at least 4 + proj varying units and at most DIST_FAST_MAX_DYN
// dynamic digits; smaller ones take the generic path.
#define DIST_FAST_PATH(i, proj) ((i) >= 4 + (proj) && (i) - 4 - (proj) <= DIST_FAST_MAX_DYN)

// Threads per block of the enumeration kernels and their minimum resident
// blocks per SM (together they set the register budget per thread).
#ifndef DIST_ENUM_THREADS
#define DIST_ENUM_THREADS 256
#endif
#ifndef DIST_ENUM_MINB
#define DIST_ENUM_MINB 2
#endif
#define DIST_ENUM_WARPS (DIST_ENUM_THREADS / 32)

// One claimable record per weight value: the first thread that finds a
// codeword of weight w (that passes the optional exclusion) writes how to
// rebuild it -- generator matrix, chosen units and the representative of each.
// WitnessSlot.gamma of a seed codeword that is not a representative of the
// plan's matrices (kept by the planner from another diagonalization).
#define DIST_SEED_GAMMA 0xFFFFFFFFu

struct WitnessSlot {
    uint32_t claim;               // 0 = free
    uint32_t gamma;               // generator matrix index (in the plan)
    uint32_t count;               // number of chosen units
    uint32_t weight;
    uint8_t unit[DIST_MAXR];      // unit indices: A-units 0..a-1, B-units a..a+b-1
    uint8_t digit[DIST_MAXR];     // representative index 0..2 of each chosen unit
};

// Device-side state of one solve.  U is the running upper bound (atomicMin),
// next_chunk the work counter of the current launch.  The single-code kernel
// also stamps its own run time (%globaltimer, ns): the complement of its
// earliest block start (kept by atomicMax, so that zero is the reset value)
// and its latest warp end; warps_done counts its finished blocks.
// next_chunk, the stamps and warps_done are reset together before every
// launch after the first.
struct Scratch {
    uint32_t U;
    uint32_t status;              // bit 1: time budget spent
    unsigned long long next_chunk;
    unsigned long long t_first_inv;
    unsigned long long t_last;
    uint32_t warps_done;
    uint32_t pad32;
    unsigned long long codewords; // (subset, representative) combinations evaluated
    WitnessSlot slot[DIST_MAXN + 1];
};
// Bytes from next_chunk to the end of warps_done (zeroed before a launch).
#define DIST_SCR_LAUNCH_RESET (4 * sizeof(unsigned long long))

// What the last block of a single-code launch writes to host-mapped memory
// when the launch asks for it, so that the host needs no copy back: the
// bound, status and codeword count after the launch, its stamps, and the
// witness slot of that bound, and the launch's sequence number (read once
// the launch has completed).
struct alignas(16) LaunchOut {
    uint32_t U;
    uint32_t status;
    unsigned long long codewords;
    unsigned long long t_first_inv;
    unsigned long long t_last;
    WitnessSlot slot;             // slot[U] (zero if U > DIST_MAXN)
    unsigned long long seq;       // the launch's EnumParams::seq
};

// Kernel run time of a launch from its stamps, seconds (0 if unset).
inline double stamps_seconds(unsigned long long t_first_inv, unsigned long long t_last) {
    if (t_last == 0 || t_first_inv == 0) return 0.0;
    const unsigned long long t0 = ~t_first_inv;
    return t_last > t0 ? 1e-9 * (double)(t_last - t0) : 0.0;
}
inline double scratch_kernel_seconds(const Scratch& s) { return stamps_seconds(s.t_first_inv, s.t_last); }

// A generator matrix as one launch sees it.
struct GammaDesc {
    uint32_t rep_off;     // word offset of its representatives in the global table buffer
    uint32_t coef_off;    // word offset of its coefficient planes
    uint32_t flag_off;    // word offset of its per-unit pivot flags
    uint32_t r0_off;      // word offset of its word-0 table ([a][3] x,z pairs)
    uint32_t r1_off;      // word offset of its word-1 table (same shape; W >= 2)
    uint32_t s_rep;       // word offset of its representatives in shared memory
    uint32_t s_r0;        // word offset of its word-0 table (U2 pairs) in shared memory
    uint32_t s_r1;        // word offset of its word-1 table in shared memory
    uint32_t s_flag;      // word offset of its pivot flags in shared memory
    uint16_t a, b;        // A-units (three representatives), B-units (one)
    int32_t gamma;        // index in the plan (witness decoding)
    int32_t t1;           // use the two-word filter when thr - P exceeds this
    uint32_t a_all;       // AND of the A-units' pivot flags
    uint32_t pad;
};

// A segment: within one step (round r of one generator matrix), the
// combinations with exactly i A-units and r-i B-units.  L_before is the lower
// bound that holds once every earlier step is complete: if U <= L_before the
// segment (and everything after it) is not needed.
struct SegDesc {
    unsigned long long NA;          // C(a, i): A-subsets
    unsigned long long NB;          // C(b, r - i): B-subsets
    unsigned long long rank0;       // this segment covers combination ranks [rank0, rank1)
    unsigned long long rank1;       //   of the NA * NB (subset pairs) of its (step, i)
    unsigned long long chunk_base;  // first global chunk index of this segment
    unsigned long long codes;       // representative choices per subset
    uint32_t i;
    uint32_t spl;                   // subsets per lane in one warp chunk
    uint16_t g;                     // GammaDesc index
    uint16_t r;
    int32_t L_before;
};

// Everything one launch needs.
struct EnumParams {
    const uint32_t* tables;             // all matrices: [u][3][2][W] reps, [u][3][2][CW] coefs
    const SegDesc* segs;                // nseg segments (copied to shared memory)
    const unsigned long long* binom;    // global [DIST_MAXU + 1][DIST_MAXR + 1], saturating
    Scratch* scr;
    uint32_t outside[DIST_MAXCW];       // coefficient bits of rows outside S
    int W, CW, proj, exclude;
    int ng, nseg;
    int brows, bcols;                   // shared binomial table shape
    uint32_t s_binom, s_segs, s_words;  // shared-memory layout (32-bit word offsets, total)
    unsigned long long nchunks;
    unsigned long long budget_ns;       // stop after this long (per block, %globaltimer); 0 = none
    int first_static;                   // 1: the first wave of chunks goes by warp index
    int two_word;                       // 0: the bound at the launch cannot reach the two-word filter
    LaunchOut* out;                     // host-mapped result of the launch, or null
    unsigned long long seq;             // written to out->seq when the result is complete
    GammaDesc g[DIST_MAXGAMMA];
};

// Whether a launch that starts with upper bound U can take the two-word
// filter: a lane takes it when thr - P > t1 for its matrix, with thr <= U
// and P >= 0 throughout the launch.
inline int enum_two_word(const EnumParams& P, uint32_t U) {
    if (P.W < 2) return 0;
    for (int g = 0; g < P.ng; g++)
        if ((long long)U > (long long)P.g[g].t1) return 1;
    return 0;
}

// One code in a multi-code launch.
struct BatchCode {
    const uint32_t* tables;             // the code's table buffer (Plan::tables on the device)
    Scratch* scr;                       // its own bound, counters and witness slots
    uint32_t outside[DIST_MAXCW];
    int32_t W, CW, proj, exclude;
    uint32_t seg0, nseg;                // its segments in BatchParams::segs
    uint32_t g0, ng;                    // its generator matrices in BatchParams::gammas
    unsigned long long nchunks;
};

// A multi-code launch: warps pick codes from `order` (codes repeated in
// proportion to their work), then pull chunks from each code's own counter.
struct BatchParams {
    const BatchCode* codes;
    const SegDesc* segs;                // SegDesc::g is relative to the code's g0
    const GammaDesc* gammas;
    const int32_t* order;               // phase 1: one chunk per entry
    const int32_t* ring;                // phase 2: codes with much work left, probed round robin
    unsigned long long* sched;          // [0] next order entry, [1] ring probe counter
    const unsigned long long* binom;    // global [DIST_MAXU + 1][DIST_MAXR + 1]
    int ncodes, norder, nring;
    unsigned long long budget_ns;       // stop after this long (per block); 0 = none
};

// What one slice of the batch engine sends to the device, at byte 0 of its
// arena: the counts, the slice's time budget and the byte offsets (from the
// arena's start) of its arrays.  The kernels of a slice take only the arena,
// so that the slice's launch sequence is one graph with fixed arguments.
struct SliceHeader {
    int32_t ncodes, norder, nring, ninit;
    unsigned long long budget_ns;       // stop after this long (per block); 0 = none
    unsigned long long off_inits, off_codes, off_segs, off_gammas, off_order, off_ring, off_sched, off_scrs,
        off_outs;
};

// Per-code scratch set-up before a multi-code launch, and the copy of a
// code's tables from the slice's upload to its device block on its first
// slice (tab_words = 0: nothing to copy).
struct BatchInit {
    Scratch* scr;
    uint32_t mode;                      // 1 = full reset + seed, 2 = restart the chunk counter
    uint32_t U0;                        // seeded upper bound (DIST_WINF = none)
    WitnessSlot slot;                   // witness of U0
    uint32_t* tab_dst;                  // the code's Plan::tables on the device
    unsigned long long tab_off;         // byte offset of the staged tables in the arena
    uint32_t tab_words;
    uint32_t pad;
};

// Per-code state read back after a multi-code launch.
struct BatchOut {
    uint32_t U, status;
    unsigned long long next_chunk, codewords;
    WitnessSlot slot;                   // slot[U] (claim = 0 if none)
};
