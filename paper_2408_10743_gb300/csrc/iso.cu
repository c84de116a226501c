// iso.cu -- the isometry method (Algorithm 3, Saved_isometry) on the GPU, a
// second algorithm beside the package method of enum.cu.  It enumerates the
// image code iso(C) in F2^{3n} with plain binary Brouwer-Zimmermann: every
// codeword of round r of a matrix is the sum of r of its rows.
//
// One launch per step (round r of matrix j).  Each block stages the matrix's
// rows, restricted to the columns outside its information set (a pivot row
// adds exactly 1 on the set, a free row 0), in shared memory; lanes walk
// rank ranges of r-subsets in revolving-door order.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/dist.h"
#include "code.h"
#include "iso.h"
#include "solve.h"
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
    const unsigned long long tw = (unsigned long long)c->dev->sms * 16ull;  // resident warps (2 x 8 per SM)
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
            // about 8 warp-chunks per resident warp, at most 2^14 subsets per lane
            unsigned long long spl = nsub / (32ull * tw * 8ull);
            spl = std::max(1ull, std::min(spl, 1ull << 14));
            P.spl = (uint32_t)spl;
            P.nchunks = (nsub + 32 * spl - 1) / (32 * spl);
            P.K = K;
            P.words = ip.G[j].words;
            P.CW = p.CW;
            P.r = r;
            P.gamma = j;
            P.exclude = p.n_stab > 0 ? 1 : 0;
            for (int w = 0; w < DIST_MAXCW; w++) P.outside[w] = p.outside[w];
            if (cudaMemsetAsync(&dscr->next_chunk, 0, sizeof(unsigned long long), st) != cudaSuccess ||
                cudaEventRecord(kit->e0, st) != cudaSuccess ||
                iso_rd_launch(P, ip.words, c->dev->sms, st) != cudaSuccess ||
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
