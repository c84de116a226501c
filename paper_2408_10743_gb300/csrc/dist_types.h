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
#define DIST_MAXSEG (DIST_MAXR + 2)
#define DIST_MAXGAMMA 16
#define DIST_WINF 0xFFFFu      // "no codeword yet" weight
#define DIST_FAST_MAX_OUTER 20 // 3^20 < 2^32: outer Gray counter fits in 32 bits

// One claimable record per weight value: the first thread that finds a
// codeword of weight w (that passes the optional exclusion) writes how to
// rebuild it -- generator matrix, chosen units and the representative of each.
struct WitnessSlot {
    uint32_t claim;               // 0 = free
    uint32_t gamma;               // generator matrix index (position in the plan)
    uint32_t count;               // number of chosen units
    uint32_t weight;
    uint8_t unit[DIST_MAXR];      // unit indices: A-units 0..a-1, B-units a..a+b-1
    uint8_t digit[DIST_MAXR];     // representative index 0..2 of each chosen unit
};

// Device-side state of one solve.  U is the running upper bound (atomicMin),
// next_chunk the work counter of the current launch.
struct Scratch {
    uint32_t U;
    uint32_t status;              // bit 0: stopped because U <= L, bit 1: deadline
    unsigned long long next_chunk;
    unsigned long long codewords; // (subset, representative) combinations evaluated
    unsigned long long pad;
    WitnessSlot slot[DIST_MAXN + 1];
};

// A segment of one enumeration step: the combinations with exactly i units
// taken from the A-units (three representatives each) and r-i from the
// B-units (one representative each).
struct SegDesc {
    unsigned long long NA;          // C(a, i): A-subsets
    unsigned long long NB;          // C(b, r - i): B-subsets
    unsigned long long chunk_base;  // first global chunk index of this segment
    unsigned long long codes;       // representative choices per subset
    uint32_t i;
    uint32_t spl;                   // subsets per lane in one warp chunk
};

// Everything one launch needs: one generator matrix, one round r.
struct EnumParams {
    const uint32_t* reps;         // [u][3][2][W] words, u = a + b, Gamma qubit order
    const uint32_t* coefs;        // [u][3][2][CW] coefficient planes (exclusion)
    const unsigned long long* binom;  // [DIST_MAXU + 1][DIST_MAXR + 1], saturating
    Scratch* scr;
    uint32_t outside[DIST_MAXCW]; // coefficient bits of rows outside S
    int a, b, W, CW, r, gamma, proj, exclude;
    int L_prev;                   // stop as soon as U <= L_prev
    int nseg;
    unsigned long long nchunks;
    unsigned long long budget_ns;     // stop after this long (per block, %globaltimer); 0 = none
    SegDesc seg[DIST_MAXSEG];
};
