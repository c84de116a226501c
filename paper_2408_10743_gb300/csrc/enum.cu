// enum.cu -- the enumeration kernel (steps S4-S5) for sm_103a.
//
// One launch runs a run of consecutive enumeration steps (round r of one
// generator matrix each), described by a segment table.  Every block stages
// the representatives of the matrices involved, their word-0 tables, the
// binomials the unranking needs and the segment table into shared memory
// (tens of KB at most); after that the kernel reads nothing from HBM except
// the running upper bound U.  Warps pull chunks of combination ranks from a
// global counter (persistent grid); every lane walks its ranks with
// walk_range(); warps sum their codeword counts with shuffles; a lane that
// finds a lighter codeword publishes it with atomicMin on U and claims the
// witness slot of that weight.  A chunk whose segment has L_before >= U is
// not needed, and neither is anything after it (L_before only grows), so the
// warp that sees it pushes the counter to the end and the grid drains.
// There is no spin-wait: the kernel ends when the chunks run out or its time
// budget is spent.
#include <cuda_runtime.h>

#include "walk.cuh"

namespace dist {

struct DevSink {
    Scratch* scr;
    __device__ __forceinline__ bool poll(uint32_t& thr, int L_before) {
        const uint32_t u = *reinterpret_cast<volatile uint32_t*>(&scr->U);
        thr = u < thr ? u : thr;
        return (int)u <= L_before;
    }
    __device__ __noinline__ void record(uint32_t w, int gamma, int count, const uint8_t* units,
                                        const uint8_t* digits) {
        if (w >= *reinterpret_cast<volatile uint32_t*>(&scr->U)) return;  // not lighter than known
        atomicMin(&scr->U, w);
        WitnessSlot* s = &scr->slot[w];
        if (atomicCAS(&s->claim, 0u, 1u) == 0u) {
            s->gamma = (uint32_t)gamma;
            s->count = (uint32_t)count;
            s->weight = w;
            for (int k = 0; k < count; k++) {
                s->unit[k] = units[k];
                s->digit[k] = digits[k];
            }
            __threadfence();
        }
    }
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

extern __shared__ __align__(16) uint32_t g_enum_smem[];

#ifndef DIST_ENUM_MINB
#define DIST_ENUM_MINB 2
#endif

__global__ void __launch_bounds__(256, DIST_ENUM_MINB) enum_kernel(const __grid_constant__ EnumParams P) {
    uint32_t* sm = g_enum_smem;
    // stage: representatives and word-0 tables of every matrix in the launch
    for (int gi = 0; gi < P.ng; gi++) {
        const GammaDesc& g = P.g[gi];
        const uint32_t* src = P.tables + g.rep_off;
        const int nw = (g.a + g.b) * 6 * P.W;
        for (int t = threadIdx.x; t < nw; t += blockDim.x) sm[g.s_rep + t] = src[t];
        U2* r0 = reinterpret_cast<U2*>(sm + g.s_r0);
        for (int t = threadIdx.x; t < g.a * 3; t += blockDim.x) {
            r0[t].x = src[(t * 2 + 0) * P.W];
            r0[t].z = src[(t * 2 + 1) * P.W];
        }
        for (int t = threadIdx.x; t < g.a + g.b; t += blockDim.x) sm[g.s_flag + t] = P.tables[g.flag_off + t];
    }
    unsigned long long* sbin = reinterpret_cast<unsigned long long*>(sm + P.s_binom);
    for (int t = threadIdx.x; t < P.brows * P.bcols; t += blockDim.x) {
        const int n = t / P.bcols, k = t - n * P.bcols;
        sbin[t] = P.binom[n * (DIST_MAXR + 1) + k];
    }
    SegDesc* ssegs = reinterpret_cast<SegDesc*>(sm + P.s_segs);
    {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(P.segs);
        uint32_t* dst = reinterpret_cast<uint32_t*>(ssegs);
        const int nw = P.nseg * (int)(sizeof(SegDesc) / 4);
        for (int t = threadIdx.x; t < nw; t += blockDim.x) dst[t] = src[t];
    }
    __syncthreads();

    DevSink sink{P.scr};
    const int lane = threadIdx.x & 31;
    const unsigned long long t_start = P.budget_ns ? global_ns() : 0ull;
    uint32_t thr = DIST_WINF;
    for (;;) {
        unsigned long long chunk = 0;
        if (lane == 0) chunk = atomicAdd(&P.scr->next_chunk, 1ull);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        if (chunk >= P.nchunks) break;
        int lo_s = 0, hi_s = P.nseg;  // last segment with chunk_base <= chunk
        while (hi_s - lo_s > 1) {
            const int mid = (lo_s + hi_s) >> 1;
            if (ssegs[mid].chunk_base <= chunk) lo_s = mid;
            else hi_s = mid;
        }
        const SegDesc sg = ssegs[lo_s];
        int skip = 0;
        if (lane == 0) {
            const uint32_t u = *reinterpret_cast<volatile uint32_t*>(&P.scr->U);
            if ((int)u <= sg.L_before) {
                skip = 1;
                atomicMax(&P.scr->next_chunk, P.nchunks);
            }
        }
        if (__shfl_sync(0xffffffffu, skip, 0)) break;
        const GammaDesc& g = P.g[sg.g];
        LaneCtx C;
        C.reps = sm + g.s_rep;
        C.r0 = reinterpret_cast<const U2*>(sm + g.s_r0);
        C.flags = sm + g.s_flag;
        C.coefs = P.tables + g.coef_off;
        C.binom = sbin;
        C.bstride = P.bcols;
        C.outside = P.outside;
        C.a = g.a;
        C.b = g.b;
        C.W = P.W;
        C.CW = P.CW;
        C.r = sg.r;
        C.gamma = g.gamma;
        C.proj = P.proj;
        C.exclude = P.exclude;
        C.L_before = sg.L_before;
        const unsigned long long total = sg.NA * sg.NB;
        const unsigned long long lo =
            (chunk - sg.chunk_base) * 32ull * sg.spl + (unsigned long long)lane * sg.spl;
        unsigned long long done = 0;
        if (lo < total) {
            const unsigned long long hi = lo + sg.spl < total ? lo + sg.spl : total;
            done = walk_range(C, sink, thr, sg, lo, hi);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) done += __shfl_xor_sync(0xffffffffu, done, off);
        int stop = 0;
        if (lane == 0) {
            if (done) atomicAdd(&P.scr->codewords, done);
            if (P.budget_ns && global_ns() - t_start > P.budget_ns) {
                atomicOr(&P.scr->status, 2u);
                atomicMax(&P.scr->next_chunk, P.nchunks);
                stop = 1;
            }
        }
        if (__shfl_sync(0xffffffffu, stop, 0)) break;
    }
}

size_t enum_smem_bytes(const EnumParams& P) { return (size_t)P.s_words * 4; }

int enum_blocks_per_sm(size_t smem) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, enum_kernel, 256, smem) != cudaSuccess)
        return 0;
    return nb;
}

cudaError_t enum_set_max_smem(size_t bytes) {
    return cudaFuncSetAttribute(enum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t enum_launch(const EnumParams& P, int grid, cudaStream_t st) {
    enum_kernel<<<grid, 256, enum_smem_bytes(P), st>>>(P);
    return cudaGetLastError();
}

}  // namespace dist
