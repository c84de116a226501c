// enum.cu -- the enumeration kernel (steps S4-S5) for sm_103a.
//
// One launch runs a run of consecutive enumeration steps (round r of one
// generator matrix each), described by a segment table.  Every block stages
// the representatives of the matrices involved, their flags, the binomials
// the unranking needs and the segment table into shared memory (tens of KB
// at most, cp.async copies), and builds the word-0/1 tables from them; after
// that the kernel reads nothing from HBM except the running upper bound U.
// Warps pull chunks of combination ranks from a global counter (persistent
// grid); every lane walks its ranks with walk_range(); a warp sums its
// codeword count with shuffles once, when it exits; a lane that finds a
// lighter codeword publishes it with atomicMin on U and claims the witness
// slot of that weight.  A chunk whose segment has L_before >= U is
// not needed, and neither is anything after it (L_before only grows), so the
// warp that sees it pushes the counter to the end and the grid drains.
// There is no spin-wait: the kernel ends when the chunks run out or its time
// budget is spent.
#include <cuda_runtime.h>

#include <vector>

#include "walk.cuh"

namespace dist {

struct DevSink {
    Scratch* scr;
    __device__ __forceinline__ bool vote_any(bool p) { return __any_sync(__activemask(), p); }
    __device__ __forceinline__ uint32_t peek() { return *reinterpret_cast<volatile uint32_t*>(&scr->U); }
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

// Asynchronous global-to-shared copies (cp.async): a block issues every copy
// of its prologue at once and waits once, so that on a cold L2 the staging
// costs about one DRAM round trip instead of one per loop step.
__device__ __forceinline__ void cp_async4(void* s, const void* g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(s)), "l"(g)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void* s, const void* g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(s)), "l"(g)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <bool kTwo>
__global__ void __launch_bounds__(DIST_ENUM_THREADS, DIST_ENUM_MINB) enum_kernel(const __grid_constant__ EnumParams P) {
    uint32_t* sm = g_enum_smem;
    if (threadIdx.x == 0) atomicMax(&P.scr->t_first_inv, ~global_ns());
    // Per-matrix lane context, read by reference from shared memory so that
    // none of it stays in registers across the inner loop.
    __shared__ LaneCtx s_ctx[DIST_MAXGAMMA];
    unsigned long long* sbin = reinterpret_cast<unsigned long long*>(sm + P.s_binom);
    if (threadIdx.x < (unsigned)P.ng) {
        const GammaDesc& g = P.g[threadIdx.x];
        LaneCtx& C = s_ctx[threadIdx.x];
        C.reps = sm + g.s_rep;
        C.r0 = reinterpret_cast<const U2*>(sm + g.s_r0);
        C.r1 = reinterpret_cast<const U2*>(sm + g.s_r1);
        C.flags = sm + g.s_flag;
        C.t1 = g.t1;
        C.a_all = g.a_all;
        C.coefs = P.tables + g.coef_off;
        C.binom = sbin;
        C.bstride = P.bcols;
        C.outside = P.outside;
        C.a = g.a;
        C.b = g.b;
        C.W = P.W;
        C.CW = P.CW;
        C.gamma = g.gamma;
        C.proj = P.proj;
        C.exclude = P.exclude;
    }
    // stage: representatives, flags and the word-0 and word-1 tables of every
    // matrix in the launch, the binomials and the segment table
    for (int gi = 0; gi < P.ng; gi++) {
        const GammaDesc& g = P.g[gi];
        const uint32_t* src = P.tables + g.rep_off;
        const int nw = (g.a + g.b) * 6 * P.W;
        for (int t = threadIdx.x; t < nw; t += blockDim.x) cp_async4(&sm[g.s_rep + t], &src[t]);
        for (int t = threadIdx.x; t < g.a + g.b; t += blockDim.x) cp_async4(&sm[g.s_flag + t], &P.tables[g.flag_off + t]);
        for (int t = threadIdx.x; t < g.a * 3; t += blockDim.x) {
            cp_async8(&sm[g.s_r0 + 2 * t], &P.tables[g.r0_off + 2 * t]);
            cp_async8(&sm[g.s_r1 + 2 * t], &P.tables[g.r1_off + 2 * t]);
        }
    }
    for (int t = threadIdx.x; t < P.brows * P.bcols; t += blockDim.x) {
        const int n = t / P.bcols, k = t - n * P.bcols;
        cp_async8(&sbin[t], &P.binom[n * (DIST_MAXR + 1) + k]);
    }
    SegDesc* ssegs = reinterpret_cast<SegDesc*>(sm + P.s_segs);
    {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(P.segs);
        uint32_t* dst = reinterpret_cast<uint32_t*>(ssegs);
        const int nw = P.nseg * (int)(sizeof(SegDesc) / 4);
        for (int t = threadIdx.x; t < nw; t += blockDim.x) cp_async4(&dst[t], &src[t]);
    }
    cp_async_wait_all();
    __syncthreads();

    DevSink sink{P.scr};
    const int lane = threadIdx.x & 31;
    const unsigned long long t_start = P.budget_ns ? global_ns() : 0ull;
    uint32_t thr = DIST_WINF;
    // Lane 0 claims the warp's next chunk, and reads U, while the current
    // chunk runs, so neither round trip stalls the warp between chunks.  The
    // skip test of a chunk therefore sees U as it was one chunk earlier; a
    // stale (larger) U only skips less, and the walk reads U afresh before
    // its first subset.  A claimed chunk is given up only where everything
    // after it is unneeded (skip) or the budget ended.
    // With first_static (set by the host when U already meets the estimate
    // of d, so that the launch is certification work and no early chunk is
    // more urgent than another) the grid's first wave of chunks is assigned:
    // warp w of block b takes chunk w * gridDim + b, consecutive chunks on
    // different SMs, and the launch does not open with every warp's atomic
    // on one counter; later claims are then the counter plus the number of
    // warps.  Otherwise every chunk is claimed, so that the chunks of the
    // early steps, where a lighter U is found, go to the warps that start
    // first.
    const unsigned long long first_off = P.first_static ? (unsigned long long)gridDim.x * (blockDim.x >> 5) : 0ull;
    unsigned long long claimed = (unsigned long long)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    uint32_t u_claim = DIST_WINF;
    if (lane == 0) {
        if (!P.first_static) claimed = atomicAdd(&P.scr->next_chunk, 1ull);
        u_claim = *reinterpret_cast<volatile uint32_t*>(&P.scr->U);
    }
    // certification work (first_static) reads U at every eighth subset
    const unsigned long long peek_mask = P.first_static ? 7ull : 0ull;
    int seg = 0;                  // chunks are claimed in increasing order
    unsigned long long done = 0;  // this lane's codewords over all its chunks
    for (;;) {
        const unsigned long long chunk = __shfl_sync(0xffffffffu, claimed, 0);
        if (chunk >= P.nchunks) break;
        const uint32_t u_now = __shfl_sync(0xffffffffu, u_claim, 0);
        if (lane == 0) {
            claimed = atomicAdd(&P.scr->next_chunk, 1ull) + first_off;
            u_claim = *reinterpret_cast<volatile uint32_t*>(&P.scr->U);
        }
        while (seg + 1 < P.nseg && ssegs[seg + 1].chunk_base <= chunk) ++seg;
        const SegDesc& sg = ssegs[seg];
        if ((int)u_now <= sg.L_before) {
            if (lane == 0) atomicMax(&P.scr->next_chunk, P.nchunks);
            break;
        }
        const LaneCtx& C = s_ctx[sg.g];
        unsigned long long lo, hi;
        if (seg_lane_range(sg, chunk, lane, lo, hi)) done += walk_range<DevSink, kTwo>(C, sink, thr, sg, lo, hi, u_now, peek_mask);
        if (P.budget_ns) {
            int stop = 0;
            if (lane == 0 && global_ns() - t_start > P.budget_ns) {
                atomicOr(&P.scr->status, 2u);
                atomicMax(&P.scr->next_chunk, P.nchunks);
                stop = 1;
            }
            if (__shfl_sync(0xffffffffu, stop, 0)) break;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) done += __shfl_xor_sync(0xffffffffu, done, off);
    if (lane == 0) {
        if (done) atomicAdd(&P.scr->codewords, done);
        atomicMax(&P.scr->t_last, global_ns());
        // the warp's updates are visible to the whole GPU before its block
        // counts itself done
        if (P.out) __threadfence();
    }
    if (P.out) {
        // the last block to finish publishes the launch's result; its loads
        // bypass L1 (every block's updates are in L2 after its fences)
        __syncthreads();
        if (threadIdx.x == 0) {
            if (atomicAdd(&P.scr->warps_done, 1u) == gridDim.x - 1u) {
                __threadfence();
                const Scratch* s = P.scr;
                const unsigned long long us = __ldcg(reinterpret_cast<const unsigned long long*>(s));
                const unsigned long long cw = __ldcg(&s->codewords);
                const unsigned long long t0 = __ldcg(&s->t_first_inv), t1 = __ldcg(&s->t_last);
                const uint32_t U = (uint32_t)us;
                const uint4* src = reinterpret_cast<const uint4*>(&s->slot[U <= DIST_MAXN ? U : 0]);
                uint4 sl[sizeof(WitnessSlot) / 16];
#pragma unroll
                for (int w = 0; w < (int)(sizeof(WitnessSlot) / 16); w++)
                    sl[w] = U <= DIST_MAXN ? __ldcg(src + w) : make_uint4(0u, 0u, 0u, 0u);
                LaunchOut* o = P.out;
                o->U = U;
                o->status = (uint32_t)(us >> 32);
                o->codewords = cw;
                o->t_first_inv = t0;
                o->t_last = t1;
                uint4* dst = reinterpret_cast<uint4*>(&o->slot);
#pragma unroll
                for (int w = 0; w < (int)(sizeof(WitnessSlot) / 16); w++) dst[w] = sl[w];
                // the host reads it after the launch has completed, when all
                // of it is visible: no system-scope fence is needed
                o->seq = P.seq;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Multi-code launch.  Each code keeps its own chunk counter and bound in its
// Scratch; the tables are read from global memory (they stay in L1/L2: a few
// KB per code).  Phase 1: every entry of the order list buys one chunk of its
// code; the list runs shortest job first and repeats each code in proportion
// to its estimated work, so newly admitted small codes get warps at once and
// large codes get many.  Phase 2: warps stay on one open code until it runs
// out, then join another from the ring of codes with much work left (small
// codes get one entry per chunk in the order list and finish in phase 1).  A
// chunk whose segment has L_before >= U retires the code (its counter is
// pushed to the end), which costs the others nothing.
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool code_open(const BatchCode& bc) {
    const unsigned long long nxt = *reinterpret_cast<volatile unsigned long long*>(&bc.scr->next_chunk);
    return nxt < bc.nchunks;
}

// Phase 2: a code that still has chunks, probing the ring (the codes with
// much work left) round robin.
__device__ int join_code(const BatchParams& P) {
    for (int probe = 0; probe < P.nring; probe++) {
        const unsigned long long k = atomicAdd(&P.sched[1], 1ull) % (unsigned long long)P.nring;
        const int c = P.ring[k];
        if (code_open(P.codes[c])) return c;
    }
    return -1;
}

// The launch's parameters, rebuilt from the slice header at the start of the
// arena (one thread per block; read from shared memory afterwards).
__device__ __forceinline__ void slice_params(const unsigned char* arena, const unsigned long long* binom,
                                             BatchParams* P) {
    const SliceHeader* H = reinterpret_cast<const SliceHeader*>(arena);
    P->codes = reinterpret_cast<const BatchCode*>(arena + H->off_codes);
    P->segs = reinterpret_cast<const SegDesc*>(arena + H->off_segs);
    P->gammas = reinterpret_cast<const GammaDesc*>(arena + H->off_gammas);
    P->order = reinterpret_cast<const int32_t*>(arena + H->off_order);
    P->ring = reinterpret_cast<const int32_t*>(arena + H->off_ring);
    P->sched = reinterpret_cast<unsigned long long*>(const_cast<unsigned char*>(arena) + H->off_sched);
    P->binom = binom;
    P->ncodes = H->ncodes;
    P->norder = H->norder;
    P->nring = H->nring;
    P->budget_ns = H->budget_ns;
}

// kTwo: with the two-word filter (as enum_kernel).  The host takes the
// instance without it unless a code of the slice has three or more words per
// plane (for up to two words the filter's registers cost more than it saves:
// 25.1 against 26.9 ms on 4096 codes of n <= 56).
template <bool kTwo>
__global__ void __launch_bounds__(DIST_ENUM_THREADS, DIST_ENUM_MINB)
    enum_batch_kernel(const unsigned char* __restrict__ arena, const unsigned long long* binom) {
    __shared__ BatchParams sP;
    __shared__ LaneCtx s_wctx[DIST_ENUM_WARPS];
    if (threadIdx.x == 0) slice_params(arena, binom, &sP);
    __syncthreads();
    const BatchParams& P = sP;
    const int lane = threadIdx.x & 31;
    const unsigned long long t_start = P.budget_ns ? global_ns() : 0ull;
    uint32_t thr = DIST_WINF;
    int cur = -1;
    bool listed = true;  // phase 1: one chunk per order-list entry
    for (;;) {
        if (listed) {
            unsigned long long k = 0;
            if (lane == 0) k = atomicAdd(&P.sched[0], 1ull);
            k = __shfl_sync(0xffffffffu, k, 0);
            if (k < (unsigned long long)P.norder) {
                const int c = P.order[k];
                if (c != cur) thr = DIST_WINF;  // another code: its own bound
                cur = c;
            } else {
                listed = false;
                cur = -1;
            }
        }
        if (!listed && cur < 0) {  // phase 2: stay on one open code until it runs out
            int c = 0;
            if (lane == 0) c = join_code(P);
            cur = __shfl_sync(0xffffffffu, c, 0);
            if (cur < 0) break;
            thr = DIST_WINF;
        }
        const BatchCode& bc = P.codes[cur];
        unsigned long long chunk = 0;
        if (lane == 0) chunk = atomicAdd(&bc.scr->next_chunk, 1ull);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        if (chunk >= bc.nchunks) {
            if (!listed) cur = -1;
            continue;
        }
        const SegDesc* segs = P.segs + bc.seg0;
        int lo_s = 0, hi_s = (int)bc.nseg;
        while (hi_s - lo_s > 1) {
            const int mid = (lo_s + hi_s) >> 1;
            if (segs[mid].chunk_base <= chunk) lo_s = mid;
            else hi_s = mid;
        }
        const SegDesc sg = segs[lo_s];
        int skip = 0;
        if (lane == 0) {
            const uint32_t u = *reinterpret_cast<volatile uint32_t*>(&bc.scr->U);
            if ((int)u <= sg.L_before) {
                skip = 1;
                atomicMax(&bc.scr->next_chunk, bc.nchunks);
            }
        }
        if (__shfl_sync(0xffffffffu, skip, 0)) {
            if (!listed) cur = -1;
            continue;
        }
        const GammaDesc& g = P.gammas[bc.g0 + sg.g];
        // The warp's lane context lives in shared memory: a local copy whose
        // address reaches the walk's cold functions would be read from local
        // memory in the hot loop.
        __syncwarp();
        LaneCtx& C = s_wctx[threadIdx.x >> 5];
        if (lane == 0) {
            C.reps = bc.tables + g.rep_off;
            C.r0 = reinterpret_cast<const U2*>(bc.tables + g.r0_off);
            C.r1 = reinterpret_cast<const U2*>(bc.tables + g.r1_off);
            C.flags = bc.tables + g.flag_off;
            C.t1 = g.t1;
            C.a_all = g.a_all;
            C.coefs = bc.tables + g.coef_off;
            C.binom = P.binom;
            C.bstride = DIST_MAXR + 1;
            C.outside = bc.outside;
            C.a = g.a;
            C.b = g.b;
            C.W = bc.W;
            C.CW = bc.CW;
            C.gamma = g.gamma;
            C.proj = bc.proj;
            C.exclude = bc.exclude;
        }
        __syncwarp();
        DevSink sink{bc.scr};
        unsigned long long lo, hi, done = 0;
        if (seg_lane_range(sg, chunk, lane, lo, hi))
            done = walk_range<DevSink, kTwo>(C, sink, thr, sg, lo, hi, sink.peek());
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) done += __shfl_xor_sync(0xffffffffu, done, off);
        int stop = 0;
        if (lane == 0) {
            if (done) atomicAdd(&bc.scr->codewords, done);
            if (P.budget_ns && global_ns() - t_start > P.budget_ns) stop = 1;
        }
        if (__shfl_sync(0xffffffffu, stop, 0)) break;
    }
}

// Scratch set-up of many codes: block i serves item i.
// Scratch set-up of the slice's new and re-planned codes (one block per code,
// the grid strides over them).
__global__ void batch_init_kernel(const unsigned char* __restrict__ arena) {
    const SliceHeader* H = reinterpret_cast<const SliceHeader*>(arena);
    const BatchInit* items = reinterpret_cast<const BatchInit*>(arena + H->off_inits);
    const int n = H->ninit;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const BatchInit it = items[i];
        if (it.tab_words) {  // the code's tables, staged in this slice's upload
            const uint32_t* src = reinterpret_cast<const uint32_t*>(arena + it.tab_off);
            for (uint32_t t = threadIdx.x; t < it.tab_words; t += blockDim.x) it.tab_dst[t] = src[t];
        }
        if (it.mode == 1) {
            uint32_t* w = reinterpret_cast<uint32_t*>(it.scr);
            for (int t = threadIdx.x; t < (int)(sizeof(Scratch) / 4); t += blockDim.x) w[t] = 0u;
            __syncthreads();
            if (threadIdx.x == 0) {
                it.scr->U = it.U0;
                if (it.U0 <= DIST_MAXN) it.scr->slot[it.U0] = it.slot;
            }
            __syncthreads();
        } else if (it.mode == 2 && threadIdx.x == 0) {
            it.scr->next_chunk = 0ull;
        }
    }
}

// Read-back of many codes: thread i gathers code i's bound, counters and the
// witness slot of its bound.
// Every code's bound, counters and witness slot into the arena's results.
__global__ void batch_gather_kernel(unsigned char* __restrict__ arena) {
    const SliceHeader* H = reinterpret_cast<const SliceHeader*>(arena);
    Scratch* const* scrs = reinterpret_cast<Scratch* const*>(arena + H->off_scrs);
    BatchOut* out = reinterpret_cast<BatchOut*>(arena + H->off_outs);
    const int n = H->ncodes;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Scratch* s = scrs[i];
        BatchOut o;
        o.U = s->U;
        o.status = s->status;
        o.next_chunk = s->next_chunk;
        o.codewords = s->codewords;
        if (o.U <= DIST_MAXN) o.slot = s->slot[o.U];
        else memset(&o.slot, 0, sizeof o.slot);
        out[i] = o;
    }
}

// The graph of one batch slice: the arena upload, the scratch set-up, the
// multi-code launch between the two timing events, the gather and the
// read-back of the results.  It is captured once per arena allocation (the
// kernels' arguments are the arena and the binomial table); before each
// replay the two copies get the slice's sizes (*h2d, *d2h: their nodes).  The
// multi-code launch (*knode) is captured without the two-word filter;
// slice_graph_set_two switches it.
cudaError_t slice_graph_build(unsigned char* d_arena, unsigned char* h_arena, const unsigned long long* binom,
                              int grid, int aux_grid, cudaEvent_t e0, cudaEvent_t e1, cudaStream_t st,
                              cudaGraph_t* graph, cudaGraphExec_t* exec, cudaGraphNode_t* h2d,
                              cudaGraphNode_t* d2h, cudaGraphNode_t* knode) {
    *graph = nullptr;
    *exec = nullptr;
    cudaError_t err = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (err != cudaSuccess) return err;
    // placeholder sizes; every replay sets the real ones
    cudaMemcpyAsync(d_arena, h_arena, sizeof(SliceHeader), cudaMemcpyHostToDevice, st);
    batch_init_kernel<<<aux_grid, 128, 0, st>>>(d_arena);
    cudaEventRecordWithFlags(e0, st, cudaEventRecordExternal);
    enum_batch_kernel<false><<<grid, DIST_ENUM_THREADS, 0, st>>>(d_arena, binom);
    cudaEventRecordWithFlags(e1, st, cudaEventRecordExternal);
    batch_gather_kernel<<<aux_grid, 128, 0, st>>>(d_arena);
    cudaMemcpyAsync(h_arena, d_arena, sizeof(SliceHeader), cudaMemcpyDeviceToHost, st);
    const cudaError_t launch_err = cudaGetLastError();
    err = cudaStreamEndCapture(st, graph);
    if (err == cudaSuccess) err = launch_err;
    if (err != cudaSuccess) {
        if (*graph) cudaGraphDestroy(*graph);
        *graph = nullptr;
        return err;
    }
    size_t nn = 0;
    err = cudaGraphGetNodes(*graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (err == cudaSuccess) err = cudaGraphGetNodes(*graph, nodes.data(), &nn);
    *h2d = *d2h = *knode = nullptr;
    for (size_t k = 0; err == cudaSuccess && k < nn; k++) {
        cudaGraphNodeType t;
        if ((err = cudaGraphNodeGetType(nodes[k], &t)) != cudaSuccess) break;
        if (t == cudaGraphNodeTypeKernel) {
            cudaKernelNodeParams kp;
            if ((err = cudaGraphKernelNodeGetParams(nodes[k], &kp)) != cudaSuccess) break;
            if (kp.func == reinterpret_cast<void*>(enum_batch_kernel<false>)) *knode = nodes[k];
            continue;
        }
        if (t != cudaGraphNodeTypeMemcpy) continue;
        cudaMemcpy3DParms mp;
        if ((err = cudaGraphMemcpyNodeGetParams(nodes[k], &mp)) != cudaSuccess) break;
        if (mp.dstPtr.ptr == static_cast<void*>(d_arena)) *h2d = nodes[k];
        else if (mp.dstPtr.ptr == static_cast<void*>(h_arena)) *d2h = nodes[k];
    }
    if (err == cudaSuccess && (!*h2d || !*d2h || !*knode)) err = cudaErrorUnknown;
    if (err == cudaSuccess) err = cudaGraphInstantiate(exec, *graph, 0);
    if (err != cudaSuccess) {
        cudaGraphDestroy(*graph);
        *graph = nullptr;
        *exec = nullptr;
    }
    return err;
}

// The slice graph's multi-code launch with (two != 0) or without the
// two-word filter, for the replays that follow.
cudaError_t slice_graph_set_two(cudaGraphExec_t exec, cudaGraphNode_t knode, int two) {
    cudaKernelNodeParams kp;
    cudaError_t err = cudaGraphKernelNodeGetParams(knode, &kp);
    if (err != cudaSuccess) return err;
    kp.func = two ? reinterpret_cast<void*>(enum_batch_kernel<true>) : reinterpret_cast<void*>(enum_batch_kernel<false>);
    return cudaGraphExecKernelNodeSetParams(exec, knode, &kp);
}

// Both instances: the occupancy of the more demanding one.
int batch_blocks_per_sm() {
    int n1 = 0, n2 = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n1, enum_batch_kernel<false>, DIST_ENUM_THREADS, 0) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n2, enum_batch_kernel<true>, DIST_ENUM_THREADS, 0) !=
            cudaSuccess)
        return 0;
    return n1 < n2 ? n1 : n2;
}

size_t enum_smem_bytes(const EnumParams& P) { return (size_t)P.s_words * 4; }

// Both instances of the kernel: the occupancy and shared-memory limits are
// those of the more demanding one.
int enum_blocks_per_sm(size_t smem) {
    int n1 = 0, n2 = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n1, enum_kernel<false>, DIST_ENUM_THREADS, smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n2, enum_kernel<true>, DIST_ENUM_THREADS, smem) != cudaSuccess)
        return 0;
    return n1 < n2 ? n1 : n2;
}

// Largest dynamic shared memory a launch may ask for: the per-block opt-in
// limit less the kernel's static shared memory (the lane contexts).
size_t enum_max_dynamic_smem(size_t optin) {
    cudaFuncAttributes a1, a2;
    if (cudaFuncGetAttributes(&a1, enum_kernel<false>) != cudaSuccess ||
        cudaFuncGetAttributes(&a2, enum_kernel<true>) != cudaSuccess)
        return 0;
    const size_t st = a1.sharedSizeBytes > a2.sharedSizeBytes ? a1.sharedSizeBytes : a2.sharedSizeBytes;
    return st >= optin ? 0 : optin - st;
}

cudaError_t enum_set_max_smem(size_t bytes) {
    const cudaError_t e = cudaFuncSetAttribute(enum_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(enum_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t enum_launch(const EnumParams& P, int grid, cudaStream_t st) {
    if (P.two_word)
        enum_kernel<true><<<grid, DIST_ENUM_THREADS, enum_smem_bytes(P), st>>>(P);
    else
        enum_kernel<false><<<grid, DIST_ENUM_THREADS, enum_smem_bytes(P), st>>>(P);
    return cudaGetLastError();
}

}  // namespace dist
