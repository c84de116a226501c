// iso.cu -- the isometry method (Algorithm 3, Saved_isometry) on the GPU, a
// second algorithm beside the package method of enum.cu.  It enumerates the
// image code iso(C) in F2^{3n} with plain binary Brouwer-Zimmermann: every
// codeword of round r of a matrix is the sum of r of its rows.
//
// One launch per step (round r of matrix j).  Each block stages the matrix's
// rows, restricted to the columns outside its information set (a pivot row
// adds exactly 1 on the set, a free row 0), in shared memory.  Large rounds
// (at most 8 rows, at least 2^18 combinations) take the split walk
// (iso_split_kernel, isosplit.cuh): the rows in two halves, every r-subset a
// product of one subset of each.  The other rounds r >= 2 walk the subsets
// in colexicographic order over a shared-memory table of all row pairs
// (iso_pair_kernel); round 1 and matrices whose pair table does not fit have
// each lane walk its own rank range in revolving-door order (iso_rd_kernel).
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "../../include/dist.h"
#include "code.h"
#include "iso.h"
#include "solve.h"
#include "isosplit.cuh"
#include "packed.cuh"
#include "rdorder.cuh"
#include "walk.cuh"

namespace dist {

namespace {

struct IsoSlot {
    uint32_t claim, count, weight, gamma;
    uint8_t rows[DIST_MAXR];
};

struct IsoScratch {
    uint32_t U;
    uint32_t status;
    unsigned long long next_chunk;
    unsigned long long codewords;
    unsigned long long pad;
    IsoSlot slot[3 * DIST_MAXN + 1];
};

struct IsoParams {
    const uint32_t* rows;    // [K][words] of this matrix
    const uint8_t* piv;      // [K]
    const uint32_t* coefs;   // [K][2][CW]
    const unsigned long long* binom;
    IsoScratch* scr;
    unsigned long long nsub;     // C(K, r)
    unsigned long long nchunks;  // warp-chunks of 32 lanes x spl subsets
    uint32_t spl;
    int K, words, CW, r, gamma, exclude;
    uint32_t outside[DIST_MAXCW];
    // split walk (iso_split_kernel): the terms of round r and their units
    SplitTerm split[kSplitMaxTerms];
    unsigned long long split_units;
    int split_nterms;
};

__device__ __noinline__ void iso_record(const IsoParams& P, uint32_t w, const uint8_t* s, uint32_t& thr) {
    if (w >= *reinterpret_cast<volatile uint32_t*>(&P.scr->U)) return;
    if (P.exclude) {  // only codewords outside S count
        uint32_t acc = 0;
        for (int q = 0; q < P.CW; q++) {
            uint32_t c0 = 0, c1 = 0;
            for (int t = 0; t < P.r; t++) {
                const uint32_t* cp = P.coefs + (size_t)s[t] * 2 * P.CW;
                c0 ^= cp[q];
                c1 ^= cp[P.CW + q];
            }
            acc |= (c0 | c1) & P.outside[q];
        }
        if (!acc) return;
    }
    thr = w;
    atomicMin(&P.scr->U, w);
    IsoSlot* sl = &P.scr->slot[w];
    if (atomicCAS(&sl->claim, 0u, 1u) == 0u) {
        sl->count = (uint32_t)P.r;
        sl->weight = w;
        sl->gamma = (uint32_t)P.gamma;
        for (int t = 0; t < P.r; t++) sl->rows[t] = s[t];
        __threadfence();
    }
}

// Full Hamming weight of the subset s (r rows) from the staged rows.
template <int WORDS>
__device__ __forceinline__ uint32_t iso_full(const uint32_t* srow, const uint8_t* spiv, const uint8_t* s, int r) {
    uint32_t v[WORDS];
#pragma unroll
    for (int w = 0; w < WORDS; w++) v[w] = 0;
    uint32_t np = 0;
    for (int t = 0; t < r; t++) {
#pragma unroll
        for (int w = 0; w < WORDS; w++) v[w] ^= srow[s[t] * WORDS + w];
        np += spiv[s[t]];
    }
#pragma unroll
    for (int w = 0; w < WORDS; w++) np += (uint32_t)__popc(v[w]);
    return np;
}

// Lane walk in revolving-door order: every step takes one row out of the
// running sum and one in, so the cost of a step does not depend on how many
// positions move (a colex carry re-adds every reset row).  The two lowest
// positions live in registers; the common step (the lowest row one up or
// down) applies one staged neighbour delta, the others go through
// rd_next_delta on the subset in local memory.
template <int WORDS>
__global__ void __launch_bounds__(256) iso_rd_kernel(const __grid_constant__ IsoParams P) {
    extern __shared__ __align__(16) uint32_t iso_smem[];
    const int K = P.K;
    uint4* sfil = reinterpret_cast<uint4*>(iso_smem);       // [K]: words 0-3
    uint4* sdel = sfil + K;                                 // [K]: words 0-3 of rows c and c + 1, XORed
    uint32_t* snp = reinterpret_cast<uint32_t*>(sdel + K);  // [K]: 1 for a pivot row
    int32_t* sdnp = reinterpret_cast<int32_t*>(snp + K);    // [K]: snp[c + 1] - snp[c]
    uint32_t* srow = reinterpret_cast<uint32_t*>(sdnp + K); // [K][WORDS]
    uint8_t* spiv = reinterpret_cast<uint8_t*>(srow + K * WORDS);
    for (int t = threadIdx.x; t < K * WORDS; t += blockDim.x) {
        const int row = t / WORDS, w = t - row * WORDS;
        srow[t] = w < P.words ? P.rows[(size_t)row * P.words + w] : 0u;
    }
    for (int t = threadIdx.x; t < K; t += blockDim.x) {
        spiv[t] = P.piv[t];
        snp[t] = P.piv[t];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < K; t += blockDim.x)
        sfil[t] = make_uint4(srow[t * WORDS], WORDS > 1 ? srow[t * WORDS + 1] : 0u,
                             WORDS > 2 ? srow[t * WORDS + 2] : 0u, WORDS > 3 ? srow[t * WORDS + 3] : 0u);
    __syncthreads();
    for (int t = threadIdx.x; t < K; t += blockDim.x) {
        const uint4 a = sfil[t], b = t + 1 < K ? sfil[t + 1] : make_uint4(0u, 0u, 0u, 0u);
        sdel[t] = make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w);
        sdnp[t] = (t + 1 < K ? (int32_t)snp[t + 1] : 0) - (int32_t)snp[t];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int r = P.r;
    volatile uint32_t* Up = &P.scr->U;
    uint32_t thr = DIST_WINF;
    for (;;) {
        unsigned long long chunk = 0;
        if (lane == 0) chunk = atomicAdd(&P.scr->next_chunk, 1ull);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        if (chunk >= P.nchunks) break;
        const unsigned long long lo = (chunk * 32ull + (unsigned long long)lane) * P.spl;
        const uint32_t left = lo < P.nsub ? (uint32_t)(min(lo + P.spl, P.nsub) - lo) : 0u;
        uint8_t s[DIST_MAXR];
        uint4 b = make_uint4(0u, 0u, 0u, 0u);
        uint32_t npb = 0;
        int c0 = 0, c1 = K;  // s[0], and s[1] (K if r < 2)
        if (left) {
            rd_unrank(P.binom, DIST_MAXR + 1, K, lo, r, s);
            for (int t = 0; t < r; t++) {
                const uint4 q = sfil[s[t]];
                b.x ^= q.x;
                b.y ^= q.y;
                b.z ^= q.z;
                b.w ^= q.w;
                npb += snp[s[t]];
            }
            c0 = s[0];
            if (r >= 2) c1 = s[1];
        }
        uint32_t u_next = *Up;
        for (uint32_t k = 0; k < P.spl; k++) {
            if ((k & 31u) == 0u) {  // the running bound, read 32 steps ahead
                thr = min(thr, u_next);
                u_next = *Up;
            }
            if (k < left) {
                uint32_t w = npb + (uint32_t)__popc(b.x) + (uint32_t)__popc(b.y);
                if (w < thr) {
                    if (WORDS > 2) w += (uint32_t)__popc(b.z) + (uint32_t)__popc(b.w);
                    if (w < thr) {
                        s[0] = (uint8_t)c0;
                        const uint32_t full = WORDS > 4 ? iso_full<WORDS>(srow, spiv, s, r) : w;
                        if (full < thr) iso_record(P, full, s, thr);
                    }
                }
                if (k + 1 < left) {
                    int o = -1;
                    if (r & 1) {
                        if (c0 + 1 < c1) o = c0++;
                    } else if (c0 > 0) {
                        o = --c0;
                    }
                    if (o >= 0) {  // the lowest row moves by one: rows o and o + 1 swap places
                        const uint4 dq = sdel[o];
                        b.x ^= dq.x;
                        b.y ^= dq.y;
                        b.z ^= dq.z;
                        b.w ^= dq.w;
                        npb = (uint32_t)((int32_t)npb + ((r & 1) ? sdnp[o] : -sdnp[o]));
                    } else {
                        s[0] = (uint8_t)c0;
                        int out, in;
                        rd_next_delta(s, r, K, &out, &in);
                        const uint4 qo = sfil[out], qi = sfil[in];
                        b.x ^= qo.x ^ qi.x;
                        b.y ^= qo.y ^ qi.y;
                        b.z ^= qo.z ^ qi.z;
                        b.w ^= qo.w ^ qi.w;
                        npb = npb - snp[out] + snp[in];
                        c0 = s[0];
                        if (r >= 2) c1 = s[1];
                    }
                }
            }
        }
        unsigned long long done = left;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) done += __shfl_xor_sync(0xffffffffu, done, off);
        if (lane == 0 && done) atomicAdd(&P.scr->codewords, done);
    }
}

// ---------------------------------------------------------------------------
// Pair-table walk (rounds r >= 2).  In colexicographic order the r-subsets
// s_1 < s_2 < ... < s_r of the rows have rank
//     sum_t C(s_t, t) = (s_1 + C(s_2, 2)) + sum_{t >= 3} C(s_t, t),
// so for a fixed "top" (s_3, ..., s_r) the subsets are consecutive and run
// through the pairs (s_1, s_2) below s_3 in the order of their pair index
// s_1 + C(s_2, 2): a prefix of length C(s_3, 2) of all C(K, 2) pairs.  Each
// block stages a table of every pair's sum on filter words 0-1 and pivot
// count, in pair-index order.  A warp takes a range of consecutive ranks;
// its lanes share the current top and take that top's pairs 32 apart, so a
// codeword is one table load, two XORs and two popcounts against the top's
// sum, and the step to the next top is the same on every lane.  Lanes idle
// only in the last pass over a top whose pair count is not a multiple of 32.
// Only a codeword whose words-0-1 bound falls below U is weighed in full.
// ---------------------------------------------------------------------------

// Largest c in [lo, hi] with C(c, t) <= R, by bisection on the binomial table.
__device__ __forceinline__ int colex_top(const unsigned long long* B, int t, unsigned long long R, int lo, int hi) {
    int a = lo, b = hi + 1;  // C(a, t) <= R < C(b, t) (C(hi + 1, t) taken as infinite)
    while (b - a > 1) {
        const int mid = (a + b) >> 1;
        if (B[mid * (DIST_MAXR + 1) + t] <= R) a = mid;
        else b = mid;
    }
    return a;
}

// Full weight of the subset (the pair from pair index p, the top (s_3..s_r)
// packed in T with its lowest element m2) and, when it beats thr, its record;
// returns the new threshold.  Inlined: as a called function it made the
// compiler keep part of the walk's state on the stack across the call site,
// one local load per top step.
template <int WORDS>
__device__ __forceinline__ uint32_t iso_pair_slow(const IsoParams& P, const uint32_t* srow, const uint8_t* spiv,
                                               uint64_t T, int m2, uint32_t p, uint32_t thr) {
    uint8_t s[DIST_MAXR];
    int c1 = 1;
    while ((unsigned)((c1 + 1) * c1 / 2) <= p) ++c1;  // C(c1 + 1, 2) > p >= C(c1, 2)
    s[0] = (uint8_t)(p - (unsigned)(c1 * (c1 - 1) / 2));
    s[1] = (uint8_t)c1;
    for (int t = 2; t < P.r; t++) s[t] = (uint8_t)pk_get(T, t - 2);
    if (P.r >= 3) s[2] = (uint8_t)m2;
    const uint32_t w = iso_full<WORDS>(srow, spiv, s, P.r);
    if (w < thr) iso_record(P, w, s, thr);
    return thr;
}

// Largest top size the pair walk keeps in one packed register.
constexpr int kIsoPairMaxTop = 8;

template <int WORDS>
__global__ void __launch_bounds__(256) iso_pair_kernel(const __grid_constant__ IsoParams P) {
    extern __shared__ __align__(16) uint32_t iso_smem[];
    const int K = P.K, r = P.r, nt = P.r - 2;  // nt: elements of the top
    const int npairs = K * (K - 1) / 2;
    uint4* spt = reinterpret_cast<uint4*>(iso_smem);         // [C(K,2)]: words 0-1 of the pair's sum, pivots
    uint4* srt = spt + npairs;                               // [K]: words 0-1 of the row, pivot
    uint4* sdt = srt + K;                                    // [K]: rows c and c + 1 XORed, pivot change
    uint32_t* srow = reinterpret_cast<uint32_t*>(sdt + K);   // [K][WORDS]
    uint8_t* spiv = reinterpret_cast<uint8_t*>(srow + K * WORDS);
    for (int t = threadIdx.x; t < K * WORDS; t += blockDim.x) {
        const int row = t / WORDS, w = t - row * WORDS;
        srow[t] = w < P.words ? P.rows[(size_t)row * P.words + w] : 0u;
    }
    for (int t = threadIdx.x; t < K; t += blockDim.x) spiv[t] = P.piv[t];
    __syncthreads();
    for (int t = threadIdx.x; t < K; t += blockDim.x)
        srt[t] = make_uint4(srow[t * WORDS], WORDS > 1 ? srow[t * WORDS + 1] : 0u, spiv[t], 0u);
    __syncthreads();
    for (int t = threadIdx.x; t < K; t += blockDim.x) {
        const uint4 a = srt[t], b = t + 1 < K ? srt[t + 1] : make_uint4(0u, 0u, 0u, 0u);
        sdt[t] = make_uint4(a.x ^ b.x, a.y ^ b.y, b.z - a.z, 0u);
    }
    for (int c1 = 1 + (int)(threadIdx.x >> 5); c1 < K; c1 += (int)(blockDim.x >> 5)) {
        const int base = c1 * (c1 - 1) / 2;
        for (int c0 = (int)(threadIdx.x & 31); c0 < c1; c0 += 32) {
            const uint4 a = srt[c0], b = srt[c1];
            spt[base + c0] = make_uint4(a.x ^ b.x, a.y ^ b.y, a.z + b.z, 0u);
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    volatile uint32_t* Up = &P.scr->U;
    uint32_t thr = DIST_WINF;
    for (;;) {
        unsigned long long chunk = 0;
        if (lane == 0) chunk = atomicAdd(&P.scr->next_chunk, 1ull);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        if (chunk >= P.nchunks) break;
        // The warp's ranks [R0, R1): every lane holds the same top; the lanes
        // take its pairs p0, p0 + 1, ... 32 apart.
        const unsigned long long R0 = chunk * 32ull * P.spl;
        const unsigned long long R1 = min(R0 + 32ull * P.spl, P.nsub);
        // the top (s_3, ..., s_r) packed, element t - 3 in bits 8(t-3)..;
        // m2 = s_3 is kept apart (the packed copy of it is refreshed only
        // where it is read), s4 = s_4 (K if there is none)
        uint64_t T = 0;
        uint32_t bx = 0, by = 0, npb = 0;
        unsigned long long R = R0;
        {
            int hi = K - 1;
            for (int t = r; t >= 3; --t) {
                const int c = colex_top(P.binom, t, R, t - 1, hi);
                T |= (uint64_t)c << (8 * (t - 3));
                R -= P.binom[c * (DIST_MAXR + 1) + t];
                const uint4 q = srt[c];
                bx ^= q.x;
                by ^= q.y;
                npb += q.z;
                hi = c - 1;
            }
        }
        uint32_t p0 = (uint32_t)R;  // pair index of rank R0 in its top
        int m2 = nt >= 1 ? pk_get(T, 0) : K;
        int s4 = nt >= 2 ? pk_get(T, 1) : K;
        uint32_t cm = (uint32_t)(m2 * (m2 - 1) / 2);
        uint32_t left = (uint32_t)(R1 - R0);  // at most 32 x 2^14
        // the running bound, prefetched and taken once at least 32 passes
        // have run since, so that the load's latency is covered (a stale,
        // larger U is still a valid threshold)
        uint32_t u_next = *Up, passes = 0;
        thr = min(thr, u_next);
        for (;;) {
            if (passes >= 32u) {
                thr = min(thr, u_next);
                u_next = *Up;
                passes = 0;
            }
            const uint32_t nh = min(cm - p0, left);
            passes += (nh + 31u) >> 5;
            // the lightest words-0-1 bound of this lane's pairs of the top,
            // with a three-way min instead of a branch per pair; the pairs
            // are weighed against thr one by one only if it beats thr (rare)
            uint32_t m = 0xFFFFu;
            uint32_t q = (uint32_t)lane;
            for (; q + 32u < nh; q += 64u) {  // two pairs per pass: two table loads in flight
                const uint32_t p = p0 + q;
                const uint4 e0 = spt[p], e1 = spt[p + 32u];
                const uint32_t w0 = e0.z + (uint32_t)__popc(bx ^ e0.x) + (uint32_t)__popc(by ^ e0.y);
                const uint32_t w1 = e1.z + (uint32_t)__popc(bx ^ e1.x) + (uint32_t)__popc(by ^ e1.y);
                m = __vimin3_u32(m, w0, w1);
            }
            if (q < nh) {
                const uint4 e = spt[p0 + q];
                m = min(m, e.z + (uint32_t)__popc(bx ^ e.x) + (uint32_t)__popc(by ^ e.y));
            }
            if (npb + m < thr) {
                for (uint32_t q2 = (uint32_t)lane; q2 < nh; q2 += 32u) {
                    const uint32_t p = p0 + q2;
                    const uint4 e = spt[p];
                    const uint32_t w = npb + e.z + (uint32_t)__popc(bx ^ e.x) + (uint32_t)__popc(by ^ e.y);
                    if (w < thr) thr = iso_pair_slow<WORDS>(P, srow, spiv, T, m2, p, thr);
                }
            }
            left -= nh;
            if (left == 0) break;
            p0 = 0;
            // the next top in colex order (the same step on every lane)
            if (m2 + 1 < s4) {  // s_3 moves up by one: C(m2 + 1, 2) = C(m2, 2) + m2
                const uint4 d = sdt[m2];
                bx ^= d.x;
                by ^= d.y;
                npb += d.z;
                cm += (uint32_t)m2;
                ++m2;
            } else {  // carry: the first s_t that can move up does, the ones below it reset
                T = pk_put(T, 0, m2);
                int t = 0;
                while (t + 1 < nt && pk_get(T, t) + 1 == pk_get(T, t + 1)) ++t;
                for (int u = 0; u < t; ++u) {
                    const uint4 qo = srt[pk_get(T, u)], qn = srt[u + 2];
                    bx ^= qo.x ^ qn.x;
                    by ^= qo.y ^ qn.y;
                    npb += qn.z - qo.z;
                    T = pk_put(T, u, u + 2);
                }
                const int c = pk_get(T, t);
                const uint4 d = sdt[c];
                bx ^= d.x;
                by ^= d.y;
                npb += d.z;
                T = pk_put(T, t, c + 1);
                m2 = pk_get(T, 0);
                s4 = nt >= 2 ? pk_get(T, 1) : K;
                cm = (uint32_t)(m2 * (m2 - 1) / 2);
            }
        }
        if (lane == 0) atomicAdd(&P.scr->codewords, R1 - R0);
    }
}

template <int WORDS>
size_t iso_pair_smem(int K) {
    return (size_t)K * (K - 1) / 2 * 16 + (size_t)K * 32 + (size_t)K * WORDS * 4 + (size_t)K + 16;
}

template <int WORDS>
cudaError_t iso_pair_launch_w(const IsoParams& P, int sms, size_t optin, cudaStream_t st, bool* used) {
    *used = false;
    const size_t smem = iso_pair_smem<WORDS>(P.K);
    if (smem > optin || P.r - 2 > kIsoPairMaxTop) return cudaSuccess;  // the caller takes the plain walk
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(iso_pair_kernel<WORDS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
        return cudaErrorUnknown;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, iso_pair_kernel<WORDS>, 256, smem) != cudaSuccess)
        return cudaErrorUnknown;
    bps = std::max(1, bps);
    const unsigned long long want = (P.nchunks + 7) / 8;
    const int grid = (int)std::min<unsigned long long>(want, (unsigned long long)sms * bps);
    iso_pair_kernel<WORDS><<<std::max(1, grid), 256, smem, st>>>(P);
    *used = true;
    return cudaGetLastError();
}

cudaError_t iso_pair_launch(const IsoParams& P, int words, int sms, size_t optin, cudaStream_t st, bool* used) {
    switch (words) {
        case 1: return iso_pair_launch_w<1>(P, sms, optin, st, used);
        case 2: return iso_pair_launch_w<2>(P, sms, optin, st, used);
        case 3: return iso_pair_launch_w<3>(P, sms, optin, st, used);
        case 4: return iso_pair_launch_w<4>(P, sms, optin, st, used);
        case 5: return iso_pair_launch_w<5>(P, sms, optin, st, used);
        case 6: return iso_pair_launch_w<6>(P, sms, optin, st, used);
        case 7: return iso_pair_launch_w<7>(P, sms, optin, st, used);
        case 8: return iso_pair_launch_w<8>(P, sms, optin, st, used);
        case 9: return iso_pair_launch_w<9>(P, sms, optin, st, used);
        case 10: return iso_pair_launch_w<10>(P, sms, optin, st, used);
        case 11: return iso_pair_launch_w<11>(P, sms, optin, st, used);
        default: return iso_pair_launch_w<12>(P, sms, optin, st, used);
    }
}

// ---------------------------------------------------------------------------
// Split walk (rounds r >= 2 of large matrices).  The rows are cut into two
// halves and round r into the products of an i-subset of one half and an
// (r - i)-subset of the other (isosplit.cuh).  A block claims a unit, stages
// the sums of its tile-side subsets in shared memory and gives each thread
// kSplitNB consecutive lane-side sums in registers; each broadcast tile
// entry is then weighed against all kSplitNB register values.
//
// The weight bound of the inner loop takes one popcount per codeword: with
// c_q = a_q XOR b_q the codeword on filter word q, popc(c_0 | c_1 | c_2) is
// at most popc(c_0) + popc(c_1) + popc(c_2), so pivot count + popc of the OR
// of words 0-2 is a lower bound on the weight.  It is tight enough to reject
// nearly every codeword (on 96 random bits it is about 28 +- 1.9 where the
// exact sum is 48 +- 4.9), and popcounts, not the XORs, are what the SM
// runs out of.  A thread keeps the lightest bound over its kSplitNB values;
// when it beats thr (rare) the values are weighed again one by one with the
// exact words-0-2 sum, and a codeword that still beats thr in full.
// ---------------------------------------------------------------------------

// Full Hamming weight of the subset s (r rows) from rows staged with
// `words` words each (run-time count: only the rare full weighing uses it).
__device__ __forceinline__ uint32_t iso_full_rt(const uint32_t* srow, int words, const uint8_t* spiv, const uint8_t* s,
                                                int r) {
    uint32_t w = 0;
    for (int t = 0; t < r; t++) w += spiv[s[t]];
    for (int q = 0; q < words; q++) {
        uint32_t v = 0;
        for (int t = 0; t < r; t++) v ^= srow[s[t] * words + q];
        w += (uint32_t)__popc(v);
    }
    return w;
}

// Full weight of the codeword (tile-side subset of rank tr, lane-side subset
// of rank lr) and, when it beats thr, its record; returns the new threshold.
// Called out of line: none of the walk's register values is live across it.
__device__ __noinline__ uint32_t iso_split_slow(const IsoParams& P, const uint32_t* srow, const uint8_t* spiv,
                                                const SplitTerm& S, unsigned long long tr, unsigned long long lr,
                                                uint32_t thr) {
    uint8_t s[DIST_MAXR];
    split_rows(P.binom, S.tile_off, S.tile_kh, S.tile_t, tr, s);
    split_rows(P.binom, S.lane_off, S.lane_kh, S.lane_t, lr, s + S.tile_t);
    const uint32_t w = iso_full_rt(srow, P.words, spiv, s, P.r);
    if (w < thr) iso_record(P, w, s, thr);
    return thr;
}

// kMode: 0, every row of the matrix has a pivot, so every r-subset has r
// pivots and the count is folded into the threshold; 1, some rows have none,
// so each register value carries its own pivot count; 2, most rows have
// none, and the pivot count no longer carries most of the bound (a matrix of
// rank 1 has one pivot row), so the bound takes a second popcount:
// popc(c_0 | c_1) + popc(c_2), about 40 +- 3.5 on random words (the OR of
// all three, 28 +- 1.9, let about one codeword in a hundred through to the
// exact weighing on such a matrix).
template <int kMode>
__global__ void __launch_bounds__(kSplitThreads, 4) iso_split_kernel(const __grid_constant__ IsoParams P) {
    constexpr bool kNp = kMode > 0;
    extern __shared__ __align__(16) uint32_t iso_smem[];
    __shared__ unsigned long long s_unit;
    const int K = P.K, words = P.words;
    SplitRow* stile = reinterpret_cast<SplitRow*>(iso_smem);  // [kSplitTile]: tile-side sums
    SplitRow* srt = stile + kSplitTile;                       // [K]: words 0-2 of each row, pivot
    SplitRow* sdt = srt + K;                                  // [K]: rows c and c + 1 XORed, pivot change
    SplitRow* sval = sdt + K;                                 // [kSplitNB][kSplitThreads]: register sets
    uint32_t* srow = reinterpret_cast<uint32_t*>(sval + kSplitNB * kSplitThreads);  // [K][words]
    uint8_t* spiv = reinterpret_cast<uint8_t*>(srow + K * words);
    const int tid = (int)threadIdx.x;
    for (int t = tid; t < K * words; t += kSplitThreads) srow[t] = P.rows[t];
    for (int t = tid; t < K; t += kSplitThreads) spiv[t] = P.piv[t];
    __syncthreads();
    for (int t = tid; t < K; t += kSplitThreads) {
        SplitRow q;
        q.x = srow[t * words];
        q.y = words > 1 ? srow[t * words + 1] : 0u;
        q.z = words > 2 ? srow[t * words + 2] : 0u;
        q.np = spiv[t];
        srt[t] = q;
    }
    __syncthreads();
    for (int t = tid; t < K; t += kSplitThreads) {
        const SplitRow a = srt[t];
        SplitRow b = {0u, 0u, 0u, 0u};
        if (t + 1 < K) b = srt[t + 1];
        SplitRow d;
        d.x = a.x ^ b.x;
        d.y = a.y ^ b.y;
        d.z = a.z ^ b.z;
        d.np = b.np - a.np;
        sdt[t] = d;
    }
    volatile uint32_t* Up = &P.scr->U;
    uint32_t thr = DIST_WINF, u_next = *Up;
    for (;;) {
        __syncthreads();  // the last unit's tile is read; s_unit is free
        if (tid == 0) s_unit = atomicAdd(&P.scr->next_chunk, 1ull);
        __syncthreads();
        const unsigned long long u = s_unit;
        if (u >= P.split_units) break;
        const SplitUnit W = split_unit(P.split, P.split_nterms, u);
        const SplitTerm& S = P.split[W.term];
        const unsigned long long t_lo = W.t_lo, t_hi = W.t_hi, l_lo = W.l_lo, l_hi = W.l_hi;
        unsigned long long q = l_lo + (unsigned long long)tid * W.per;
        const unsigned long long q_end = min(l_hi, q + W.per);
        uint64_t T = 0;
        SplitRow lv = {0u, 0u, 0u, 0u};
        if (q < q_end) split_unrank(P.binom, srt, S.lane_off, S.lane_kh, S.lane_t, q, &T, &lv);
        const int ntiles = (int)((t_hi - t_lo + kSplitTile - 1) / kSplitTile);
        if (ntiles == 1) {  // a short tile side: staged once for all register sets
            const unsigned long long tr = t_lo + (unsigned long long)tid;
            if (tr < t_hi) {
                uint64_t TT;
                split_unrank(P.binom, srt, S.tile_off, S.tile_kh, S.tile_t, tr, &TT, &stile[tid]);
            }
            __syncthreads();
        }
        for (uint32_t gi = 0; gi < S.groups; ++gi) {
            // this thread's next kSplitNB lane-side sums, stepped in a loop
            // through its own slots of shared memory (the step's registers
            // are not live beside the register set)
            const unsigned long long qg = q;  // rank of register value 0
            for (int j = 0; j < kSplitNB; j++) {
                SplitRow v = lv;
                if (q < q_end) {
                    ++q;
                    if (q < q_end) split_next(srt, sdt, S.lane_off, S.lane_t, &T, &lv);
                } else {  // no value: all-zero words, and a pivot count no threshold accepts
                    v.x = v.y = v.z = 0u;
                    v.np = DIST_WINF;
                }
                sval[j * kSplitThreads + tid] = v;
            }
            for (int tt = 0; tt < ntiles; ++tt) {
                const unsigned long long base = t_lo + (unsigned long long)tt * kSplitTile;
                const int len = (int)min((unsigned long long)kSplitTile, t_hi - base);
                if (ntiles > 1) {  // one register set per thread; the tile range staged piece by piece
                    __syncthreads();
                    if (tid < len) {
                        uint64_t TT;
                        split_unrank(P.binom, srt, S.tile_off, S.tile_kh, S.tile_t, base + (unsigned long long)tid,
                                     &TT, &stile[tid]);
                    }
                    __syncthreads();
                }
                // the running bound, read one piece ahead (a stale, larger U
                // is still a valid threshold)
                thr = min(thr, u_next);
                u_next = *Up;
                // without free rows every codeword has r pivots: the bound
                // on words 0-2 must stay below thr - r
                const uint32_t thr_w = kNp ? thr : (thr > (uint32_t)P.r ? thr - (uint32_t)P.r : 0u);
                int k = 0;
                for (;;) {
                    // the register set, (re)loaded from its slots: it is not
                    // live across the rare weighing below
                    uint32_t vx[kSplitNB], vy[kSplitNB], vz[kSplitNB], vn[kSplitNB];
#pragma unroll
                    for (int j = 0; j < kSplitNB; j++) {
                        const SplitRow v = sval[j * kSplitThreads + tid];
                        vx[j] = v.x;
                        vy[j] = v.y;
                        vz[j] = v.z;
                        vn[j] = kNp ? v.np : 0u;
                    }
                    for (; k < len; ++k) {
                        const SplitRow a = stile[k];
                        uint32_t m = DIST_WINF;
#pragma unroll
                        for (int j = 0; j < kSplitNB; j += 2) {
                            uint32_t w0, w1;
                            if (kMode == 2) {
                                w0 = (uint32_t)__popc((a.x ^ vx[j]) | (a.y ^ vy[j])) + (uint32_t)__popc(a.z ^ vz[j]) +
                                     vn[j];
                                w1 = (uint32_t)__popc((a.x ^ vx[j + 1]) | (a.y ^ vy[j + 1])) +
                                     (uint32_t)__popc(a.z ^ vz[j + 1]) + vn[j + 1];
                            } else {
                                w0 = (uint32_t)__popc((a.x ^ vx[j]) | (a.y ^ vy[j]) | (a.z ^ vz[j])) + vn[j];
                                w1 = (uint32_t)__popc((a.x ^ vx[j + 1]) | (a.y ^ vy[j + 1]) | (a.z ^ vz[j + 1])) +
                                     vn[j + 1];
                            }
                            m = __vimin3_u32(m, w0, w1);
                        }
                        if (kNp) m += a.np;
                        if (m < thr_w) break;
                    }
                    if (k >= len) break;
                    // entry k meets a register value whose bound beats thr
                    // (rare): the exact words-0-2 weight of each, and the
                    // full weight of any that still beats it
                    const SplitRow a = stile[k];
#pragma unroll 1
                    for (int j = 0; j < kSplitNB; j++) {
                        const SplitRow v = sval[j * kSplitThreads + tid];
                        const uint32_t w = a.np + v.np + (uint32_t)__popc(a.x ^ v.x) + (uint32_t)__popc(a.y ^ v.y) +
                                           (uint32_t)__popc(a.z ^ v.z);
                        if (w < thr && qg + (unsigned long long)j < q_end)
                            thr = iso_split_slow(P, srow, spiv, S, base + (unsigned long long)k,
                                                 qg + (unsigned long long)j, thr);
                    }
                    ++k;
                }
            }
        }
        if (tid == 0) atomicAdd(&P.scr->codewords, (t_hi - t_lo) * (l_hi - l_lo));
    }
}

size_t iso_split_smem(int K, int words) {
    return (size_t)kSplitTile * 16 + (size_t)K * 32 + (size_t)kSplitNB * kSplitThreads * 16 + (size_t)K * words * 4 +
           (size_t)K + 16;
}

template <int kMode>
cudaError_t iso_split_launch_t(const IsoParams& P, int sms, size_t optin, cudaStream_t st, bool* used) {
    *used = false;
    const size_t smem = iso_split_smem(P.K, P.words);
    if (smem > optin || P.split_units == 0) return cudaSuccess;  // the caller takes another walk
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(iso_split_kernel<kMode>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
        return cudaErrorUnknown;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, iso_split_kernel<kMode>, kSplitThreads, smem) !=
        cudaSuccess)
        return cudaErrorUnknown;
    bps = std::max(1, bps);
    const int grid = (int)std::min<unsigned long long>(P.split_units, (unsigned long long)sms * bps);
    iso_split_kernel<kMode><<<std::max(1, grid), kSplitThreads, smem, st>>>(P);
    *used = true;
    return cudaGetLastError();
}

// free_rows: rows of the matrix without a pivot, of K.
cudaError_t iso_split_launch(const IsoParams& P, int free_rows, int sms, size_t optin, cudaStream_t st, bool* used) {
    if (free_rows == 0) return iso_split_launch_t<0>(P, sms, optin, st, used);
    if (4 * free_rows <= P.K) return iso_split_launch_t<1>(P, sms, optin, st, used);
    return iso_split_launch_t<2>(P, sms, optin, st, used);
}

template <int WORDS>
cudaError_t iso_rd_launch_w(const IsoParams& P, int sms, cudaStream_t st) {
    const size_t smem = (size_t)P.K * 40 + (size_t)P.K * WORDS * 4 + (size_t)P.K + 16;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, iso_rd_kernel<WORDS>, 256, smem) != cudaSuccess)
        return cudaErrorUnknown;
    bps = std::max(1, bps);
    const unsigned long long want = (P.nchunks + 7) / 8;
    const int grid = (int)std::min<unsigned long long>(want, (unsigned long long)sms * bps);
    iso_rd_kernel<WORDS><<<std::max(1, grid), 256, smem, st>>>(P);
    return cudaGetLastError();
}

cudaError_t iso_rd_launch(const IsoParams& P, int words, int sms, cudaStream_t st) {
    switch (words) {
        case 1: return iso_rd_launch_w<1>(P, sms, st);
        case 2: return iso_rd_launch_w<2>(P, sms, st);
        case 3: return iso_rd_launch_w<3>(P, sms, st);
        case 4: return iso_rd_launch_w<4>(P, sms, st);
        case 5: return iso_rd_launch_w<5>(P, sms, st);
        case 6: return iso_rd_launch_w<6>(P, sms, st);
        case 7: return iso_rd_launch_w<7>(P, sms, st);
        case 8: return iso_rd_launch_w<8>(P, sms, st);
        case 9: return iso_rd_launch_w<9>(P, sms, st);
        case 10: return iso_rd_launch_w<10>(P, sms, st);
        case 11: return iso_rd_launch_w<11>(P, sms, st);
        default: return iso_rd_launch_w<12>(P, sms, st);
    }
}

unsigned long long binom_u64(int n, int k) {
    if (k < 0 || k > n) return 0;
    unsigned long long c = 1;
    for (int i = 1; i <= k; i++) {
        const unsigned __int128 t = (unsigned __int128)c * (unsigned long long)(n - k + i);
        c = (unsigned long long)(t / (unsigned long long)i);
        if (c >> 62) return ~0ull;
    }
    return c;
}

}  // namespace

}  // namespace dist

using namespace dist;

namespace {
std::atomic<int> g_iso_walk{0};
constexpr unsigned long long kSplitMinCombinations = 1ull << 18;
}  // namespace

extern "C" int dist_set_iso_walk(int mode) {
    if (mode < 0 || mode > 2) return DIST_EINVAL;
    g_iso_walk.store(mode);
    return DIST_OK;
}

extern "C" int dist_get_iso_walk(void) { return g_iso_walk.load(); }

extern "C" int dist_solve_isometry(dist_code* c, dist_result* out, void* cuda_stream) {
    if (!c || !out) return DIST_EINVAL;
    if (c->in_batch) return DIST_EBUSY;
    memset(out, 0, sizeof *out);
    const double t0 = wall_now();
    int prev_dev = -1;  // run on the code's device, restore the caller's after
    if (cudaGetDevice(&prev_dev) != cudaSuccess) return DIST_ECUDA;
    if (prev_dev != c->dev->device && cudaSetDevice(c->dev->device) != cudaSuccess) return DIST_ECUDA;
    struct Restore {
        int dev, prev;
        ~Restore() {
            if (prev != dev) cudaSetDevice(prev);
        }
    } restore{c->dev->device, prev_dev};
    const Plan& p = c->plan;
    if (p.n_stab > 0 && p.s_rank == p.k_eff) return DIST_EZERO;
    IsoPlan ip;
    int rc = map_plan_rc(iso_build(p, &ip));
    if (rc) return rc;
    const int m = (int)ip.G.size(), K = ip.K;
    // device image: every matrix's rows, pivot flags and coefficients, then
    // the scratch
    std::vector<size_t> o_rows(m), o_piv(m), o_coef(m);
    size_t bytes = 0;
    for (int j = 0; j < m; j++) {
        o_rows[j] = bytes;
        bytes += ip.G[j].rows.size() * 4;
        o_piv[j] = bytes;
        bytes = align256(bytes + (size_t)K);
        o_coef[j] = bytes;
        bytes += (size_t)K * 2 * p.CW * 4;
        bytes = align256(bytes);
    }
    const size_t o_scr = bytes;
    bytes += sizeof(IsoScratch);
    std::vector<unsigned char> img(bytes, 0);
    for (int j = 0; j < m; j++) {
        const IsoGamma& G = ip.G[j];
        memcpy(&img[o_rows[j]], G.rows.data(), G.rows.size() * 4);
        memcpy(&img[o_piv[j]], G.piv.data(), (size_t)K);
        uint32_t* cp = reinterpret_cast<uint32_t*>(&img[o_coef[j]]);
        for (int i = 0; i < K; i++)
            for (int q = 0; q < 2; q++)
                for (int w = 0; w < p.CW; w++) cp[((size_t)i * 2 + q) * p.CW + w] = G.coef[i].p[q][w];
    }
    IsoScratch* hs = reinterpret_cast<IsoScratch*>(&img[o_scr]);
    hs->U = (uint32_t)std::min<int>(ip.u0, DIST_WINF);
    if (ip.u0 < (int)DIST_WINF) {  // the lightest row is a codeword: seed U with it
        IsoSlot& sl = hs->slot[ip.u0];
        sl.claim = 1;
        sl.count = 1;
        sl.weight = (uint32_t)ip.u0;
        sl.gamma = (uint32_t)ip.u0_g;
        sl.rows[0] = (uint8_t)ip.u0_row;
    }
    void* d_block = nullptr;
    size_t cap = 0;
    rc = block_acquire(c->dev, bytes, &d_block, &cap);
    if (rc) return rc;
    SolveKit* kit = nullptr;
    rc = kit_acquire(c->dev, &kit);
    if (rc) {
        block_release(c->dev, d_block, cap);
        return rc;
    }
    cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : kit->stream;
    unsigned char* db = static_cast<unsigned char*>(d_block);
    IsoScratch* dscr = reinterpret_cast<IsoScratch*>(db + o_scr);
    int status = DIST_OK;
    uint32_t U = hs->U;
    unsigned long long codewords = 0, launches = 0;
    double gpu_s = 0;
    int L = iso_lower_bound(ip, 0, m - 1), rounds = 0;
    if (cudaMemcpyAsync(db, img.data(), bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) status = DIST_ECUDA;
    const unsigned long long tw = (unsigned long long)c->dev->sms * 32ull;  // resident warps (4 x 8 per SM)
    const int walk = g_iso_walk.load(std::memory_order_relaxed);
    std::vector<unsigned long long> hbinom((DIST_MAXU + 1) * (DIST_MAXR + 1));
    binom_table(hbinom.data());
    // rounds r >= 2 take the split walk where it applies, else the pair-table
    // walk where its table fits in shared memory; round 1 and the rest the
    // revolving-door walk
    auto launch_step = [&](const IsoParams& P) -> cudaError_t {
        if (P.split_units) {
            bool used = false;
            const cudaError_t e = iso_split_launch(P, ip.G[P.gamma].f, c->dev->sms, c->dev->smem_optin, st, &used);
            if (e != cudaSuccess || used) return e;
        }
        if (P.r >= 2) {
            bool used = false;
            const cudaError_t e = iso_pair_launch(P, ip.words, c->dev->sms, c->dev->smem_optin, st, &used);
            if (e != cudaSuccess || used) return e;
        }
        return iso_rd_launch(P, ip.words, c->dev->sms, st);
    };
    for (int r = 1; status == DIST_OK && r <= std::min(K, DIST_MAXR); r++) {
        for (int j = 0; j < m; j++) {
            if (U != DIST_WINF && L >= (int)U) goto certified;
            const unsigned long long nsub = binom_u64(K, r);
            if (nsub == ~0ull) {
                status = DIST_ERANGE;
                break;
            }
            IsoParams P;
            memset(&P, 0, sizeof P);
            P.rows = reinterpret_cast<const uint32_t*>(db + o_rows[j]);
            P.piv = db + o_piv[j];
            P.coefs = reinterpret_cast<const uint32_t*>(db + o_coef[j]);
            P.binom = c->dev->d_binom;
            P.scr = dscr;
            P.nsub = nsub;
            // about 32 warp-chunks per resident warp, at most 2^11 subsets per
            // lane (about half a millisecond of a warp), so that the last
            // chunks leave little of the GPU idle
            unsigned long long spl = nsub / (32ull * tw * 32ull);
            spl = std::max(1ull, std::min(spl, 1ull << 11));
            P.spl = (uint32_t)spl;
            P.nchunks = (nsub + 32 * spl - 1) / (32 * spl);
            P.K = K;
            P.words = ip.G[j].words;
            P.CW = p.CW;
            P.r = r;
            P.gamma = j;
            P.exclude = p.n_stab > 0 ? 1 : 0;
            for (int w = 0; w < DIST_MAXCW; w++) P.outside[w] = p.outside[w];
            if (r >= 2 && walk != 2 && (walk == 1 || nsub >= kSplitMinCombinations)) {
                // units of about 1/16 of a resident block's share of the round
                unsigned long long target = nsub / ((unsigned long long)c->dev->sms * 4ull * 16ull);
                target = std::max(1ull << 15, std::min(target, 1ull << 21));
                SplitPlan sp;
                if (split_plan(K, r, target, hbinom.data(), &sp)) {
                    for (int e = 0; e < sp.nterms; e++) P.split[e] = sp.term[e];
                    P.split_nterms = sp.nterms;
                    P.split_units = sp.units;
                }
            }
            if (cudaMemsetAsync(&dscr->next_chunk, 0, sizeof(unsigned long long), st) != cudaSuccess ||
                cudaEventRecord(kit->e0, st) != cudaSuccess ||
                launch_step(P) != cudaSuccess ||
                cudaEventRecord(kit->e1, st) != cudaSuccess ||
                cudaMemcpyAsync(hs, dscr, 32, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                status = DIST_ECUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, kit->e0, kit->e1);
            gpu_s += ms * 1e-3;
            launches++;
            U = hs->U;
            codewords = hs->codewords;
            rounds = r;
            L = iso_lower_bound(ip, r, j);
            if (L == (int)DIST_WINF) goto certified;  // a matrix enumerated completely
        }
        if (r == DIST_MAXR && status == DIST_OK) status = DIST_ERANGE;
    }
certified:
    if (status == DIST_OK) {
        if (U == DIST_WINF) {
            status = DIST_EZERO;
        } else if (cudaMemcpyAsync(&hs->slot[U], &dscr->slot[U], sizeof(IsoSlot), cudaMemcpyDeviceToHost, st) !=
                       cudaSuccess ||
                   cudaStreamSynchronize(st) != cudaSuccess) {
            status = DIST_ECUDA;
        } else {
            const IsoSlot& sl = hs->slot[U];
            if (sl.claim == 0 || iso_decode(p, ip, (int)sl.gamma, sl.rows, (int)sl.count, (int)U, out->witness,
                                            out->coeffs) != P_OK)
                status = DIST_EINTERNAL;
            out->d = (int)U / 2;
            out->lower = out->d;
        }
    }
    if (status != DIST_OK) cudaStreamSynchronize(st);
    kit_release(c->dev, kit);
    block_release(c->dev, d_block, cap);
    out->rounds = rounds;
    out->k_eff = p.k_eff;
    out->n_gamma = m;
    out->codewords = codewords;
    out->gpu_seconds = gpu_s;
    out->launches = launches;
    out->seconds = wall_now() - t0;
    out->status = status;
    return status;
}
