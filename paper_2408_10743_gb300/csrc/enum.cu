// enum.cu -- the enumeration kernel (steps S4-S5) for sm_103a.
//
// One launch = one round r of one generator matrix.  The matrix's
// representatives (a few KB) are staged once per block into shared memory;
// after that the kernel reads nothing from HBM except the running upper bound
// U.  Warps pull chunks of combination ranks from a global counter
// (persistent grid, one block per resident slot), every lane walks its
// ranks with walk_range(), warps sum their codeword counts with shuffles, and
// a lane that finds a lighter codeword publishes it with atomicMin on U and
// claims the witness slot of that weight.  Every lane re-reads U once per
// subset, so the whole grid stops shortly after U drops to the bound already
// in force.  There is no spin-wait anywhere: the kernel ends when the chunks
// run out, when U <= L, or when its time budget is spent.
#include <cuda_runtime.h>

#include "walk.cuh"

namespace dist {

struct DevSink {
    Scratch* scr;
    int L_prev;
    __device__ __forceinline__ bool poll(uint32_t& thr) {
        const uint32_t u = *reinterpret_cast<volatile uint32_t*>(&scr->U);
        thr = u < thr ? u : thr;
        return (int)u <= L_prev;
    }
    __device__ __noinline__ void record(uint32_t w, int gamma, int count, const uint8_t* units,
                                        const uint8_t* digits) {
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

__global__ void __launch_bounds__(256, 2) enum_kernel(const __grid_constant__ EnumParams P) {
    const int u = P.a + P.b;
    const int nrep = u * 3 * 2 * P.W;
    uint32_t* s_reps = g_enum_smem;
    U2* s_r0 = reinterpret_cast<U2*>(g_enum_smem + ((nrep + 1) & ~1));
    for (int t = threadIdx.x; t < nrep; t += blockDim.x) s_reps[t] = P.reps[t];
    for (int t = threadIdx.x; t < P.a * 3; t += blockDim.x) {
        s_r0[t].x = P.reps[(t * 2 + 0) * P.W];
        s_r0[t].z = P.reps[(t * 2 + 1) * P.W];
    }
    __syncthreads();

    LaneCtx C;
    C.reps = s_reps;
    C.r0 = s_r0;
    C.coefs = P.coefs;
    C.binom = P.binom;
    C.outside = P.outside;
    C.a = P.a;
    C.b = P.b;
    C.W = P.W;
    C.CW = P.CW;
    C.r = P.r;
    C.gamma = P.gamma;
    C.proj = P.proj;
    C.exclude = P.exclude;
    DevSink sink{P.scr, P.L_prev};

    const int lane = threadIdx.x & 31;
    const unsigned long long t_start = P.budget_ns ? global_ns() : 0ull;
    uint32_t thr = DIST_WINF;
    for (;;) {
        unsigned long long chunk = 0;
        if (lane == 0) chunk = atomicAdd(&P.scr->next_chunk, 1ull);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        if (chunk >= P.nchunks) break;
        int sgi = 0;
        while (sgi + 1 < P.nseg && P.seg[sgi + 1].chunk_base <= chunk) ++sgi;
        const SegDesc sg = P.seg[sgi];
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
            const uint32_t uu = *reinterpret_cast<volatile uint32_t*>(&P.scr->U);
            stop = (int)uu <= P.L_prev;
            if (!stop && P.budget_ns && global_ns() - t_start > P.budget_ns) {
                atomicOr(&P.scr->status, 2u);
                stop = 1;
            }
        }
        if (__shfl_sync(0xffffffffu, stop, 0)) break;
    }
}

size_t enum_smem_bytes(const EnumParams& P) {
    const size_t nrep = (size_t)(P.a + P.b) * 3 * 2 * P.W;
    return ((nrep + 1) & ~(size_t)1) * 4 + (size_t)P.a * 3 * sizeof(U2);
}

int enum_blocks_per_sm(size_t smem) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, enum_kernel, 256, smem) != cudaSuccess)
        return 0;
    return nb;
}

cudaError_t enum_launch(const EnumParams& P, int max_blocks, cudaStream_t st) {
    const size_t smem = enum_smem_bytes(P);
    unsigned long long want = (P.nchunks + 7) / 8;  // eight warps per block
    if (want < 1) want = 1;
    const int grid = (int)(want < (unsigned long long)max_blocks ? want : (unsigned long long)max_blocks);
    enum_kernel<<<grid, 256, smem, st>>>(P);
    return cudaGetLastError();
}

}  // namespace dist
