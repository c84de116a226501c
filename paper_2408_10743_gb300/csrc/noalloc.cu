// noalloc.cu -- dist_solve_noalloc: the whole solve without allocating any
// device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or under a strict device-memory budget, processes
// that must never grow their device footprint after start-up, or code paths
// where an allocation could block or fail at the wrong moment.  For them this
// entry point keeps every byte of device scratch the enumeration kernel needs
// -- the running bound and witness slots, the segment table, the binomial
// rows and the generator-matrix tables -- in one file-scope array of a fixed
// size (DIST_NOALLOC_MAX_BYTES).  Every GPU that loads the library holds that
// array until the process exits.  Host code cannot use the array's name as a
// device address, so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and passes the pointer to
// the kernel.
//
// Nothing here calls cudaMalloc, cudaFree, cudaMallocHost, a stream or event
// constructor, or any allocating library routine; the host planner uses
// ordinary heap memory.  Calls share the array: each call clears the parts
// that must start at zero, and two calls whose work overlaps on the GPU
// (different streams, or different host threads) race on it.
#include <cuda_runtime.h>
#include <stddef.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "../../include/dist.h"
#include "plan.h"
#include "solve.h"

namespace dist {
cudaError_t enum_launch(const EnumParams& P, int grid, cudaStream_t st);
size_t enum_smem_bytes(const EnumParams& P);
int enum_blocks_per_sm(size_t smem);
size_t enum_max_dynamic_smem(size_t optin);
cudaError_t enum_set_max_smem(size_t bytes);
}  // namespace dist

using namespace dist;

static __device__ __align__(256) unsigned char g_noalloc_scratch[DIST_NOALLOC_MAX_BYTES];

namespace {

struct NoAllocDevice {
    bool ready = false;
    unsigned char* base = nullptr;  // device address of g_noalloc_scratch
    int sms = 0;
    int blocks_per_sm = 0;
    size_t smem_optin = 0;
};

std::mutex g_na_mu;
NoAllocDevice g_na_dev[64];

// One-time set-up per device, with that device current.
int noalloc_device(NoAllocDevice** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return DIST_ECUDA;
    std::lock_guard<std::mutex> lk(g_na_mu);
    NoAllocDevice& d = g_na_dev[dev];
    if (!d.ready) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DIST_ECUDA;
        int optin = 0;
        if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            return DIST_ECUDA;
        d.smem_optin = enum_max_dynamic_smem((size_t)optin);
        if (d.smem_optin == 0 || enum_set_max_smem(d.smem_optin) != cudaSuccess) return DIST_ECUDA;
        d.blocks_per_sm = enum_blocks_per_sm(16 * 1024);
        if (d.blocks_per_sm < 1) return DIST_ECUDA;
        d.base = (unsigned char*)p;
        d.ready = true;
    }
    *out = &d;
    return DIST_OK;
}

// Layout of the array for one code (byte offsets, 256-byte aligned).
struct Layout {
    size_t scr, segs, binom, tables, total;
    int brows;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

Layout layout_for(const Plan& p) {
    Layout L;
    int maxrow = 1;
    for (const Gamma& G : p.gammas) maxrow = std::max(maxrow, std::max((int)G.A.size(), (int)G.B.size()));
    L.brows = maxrow + 1;
    L.scr = 0;
    L.segs = align256(L.scr + sizeof(Scratch));
    L.binom = align256(L.segs + DIST_MAXSEG * sizeof(SegDesc));
    L.tables = align256(L.binom + (size_t)L.brows * (DIST_MAXR + 1) * sizeof(unsigned long long));
    L.total = L.tables + p.tables.size() * sizeof(uint32_t);
    return L;
}

// Executor of solve_loop that works only inside the static array.
struct NoAllocExec {
    const Plan& p;
    NoAllocDevice* d;
    Layout L;
    cudaStream_t st;
    unsigned long long nl = 0;
    uint32_t U_host = DIST_WINF;  // the device's U as of the last copy or read-back
    Scratch* scr() const { return (Scratch*)(d->base + L.scr); }
    int reset() {
        if (cudaMemsetAsync(scr(), 0, sizeof(Scratch), st) != cudaSuccess) return DIST_ECUDA;
        if (cudaMemsetAsync(scr(), 0xFF, 2, st) != cudaSuccess) return DIST_ECUDA;  // U = 0xFFFF
        U_host = DIST_WINF;
        return DIST_OK;
    }
    int seed(uint32_t U0, const WitnessSlot& s) {
        if (cudaMemcpyAsync(&scr()->U, &U0, sizeof U0, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(&scr()->slot[U0], &s, sizeof s, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return DIST_ECUDA;
        U_host = U0;
        return DIST_OK;
    }
    int target_warps() const { return d->sms * d->blocks_per_sm * DIST_ENUM_WARPS; }
    double gpu_s = 0.0;
    double gpu_seconds() const { return gpu_s; }
    unsigned long long launches() const { return nl; }
    int run(const LaunchPlan& lp, double deadline_wall, StepResult* out) {
        EnumParams ep;
        plan_params(p, lp, &ep);
        ep.tables = (const uint32_t*)(d->base + L.tables);
        ep.segs = (const SegDesc*)(d->base + L.segs);
        ep.binom = (const unsigned long long*)(d->base + L.binom);
        ep.scr = scr();
        // U already at the random-code estimate of d: certification work
        // (the same first-wave rule as dist_solve)
        ep.first_static = U_host <= (uint32_t)p.d_est ? 1 : 0;
        ep.two_word = enum_two_word(ep, U_host);
        if (deadline_wall > 0) {
            double left = deadline_wall - wall_now();
            ep.budget_ns = left > 1e-3 ? (unsigned long long)(left * 1e9) : 1000000ull;
        }
        if (lp.brows > L.brows) return DIST_EINTERNAL;
        const size_t smem = enum_smem_bytes(ep);
        if (smem > d->smem_optin) return DIST_ERANGE;
        const int bps = enum_blocks_per_sm(smem);
        if (bps < 1) return DIST_ECUDA;
        unsigned long long want = (lp.nchunks + DIST_ENUM_WARPS - 1) / DIST_ENUM_WARPS;
        if (want < 1) want = 1;
        const unsigned long long cap = (unsigned long long)d->sms * (unsigned long long)bps;
        const int grid = (int)(want < cap ? want : cap);
        if (cudaMemcpyAsync(d->base + L.segs, lp.segs.data(), lp.segs.size() * sizeof(SegDesc),
                            cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemsetAsync(&scr()->next_chunk, 0, DIST_SCR_LAUNCH_RESET, st) != cudaSuccess)
            return DIST_ECUDA;
        if (enum_launch(ep, grid, st) != cudaSuccess) return DIST_ECUDA;
        nl++;
        // the fields before the witness slots: bound, status, stamps, count
        Scratch head;
        if (cudaMemcpyAsync(&head, scr(), offsetof(Scratch, slot), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return DIST_ECUDA;
        out->U = head.U;
        U_host = out->U;
        out->status = head.status;
        out->codewords = head.codewords;
        gpu_s += scratch_kernel_seconds(head);
        return DIST_OK;
    }
    int read_slot(uint32_t w, WitnessSlot* s) {
        if (w > DIST_MAXN) return DIST_EINTERNAL;
        if (cudaMemcpyAsync(s, &scr()->slot[w], sizeof *s, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return DIST_ECUDA;
        return DIST_OK;
    }
};

int map_rc(int rc) {
    switch (rc) {
        case P_OK: return DIST_OK;
        case P_EZERO: return DIST_EZERO;
        case P_ENOMEM: return DIST_ENOMEM;
        case P_ERANGE: return DIST_ERANGE;
        default: return DIST_EINVAL;
    }
}

}  // namespace

extern "C" int dist_solve_noalloc(const uint8_t* generator, int n, int K, int field, int n_stab,
                                  dist_result* out, void* cuda_stream) {
    if (!generator || !out) return DIST_EINVAL;
    Plan p;
    int rc = map_rc(plan_build(generator, n, K, field, &p));
    if (rc) return rc;
    if (n_stab) {
        rc = map_rc(plan_set_exclude(&p, n_stab));
        if (rc) return rc;
    }
    const Layout L = layout_for(p);
    if (L.total > DIST_NOALLOC_MAX_BYTES) return DIST_ERANGE;  // does not fit the static array
    NoAllocDevice* d = nullptr;
    rc = noalloc_device(&d);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    std::vector<unsigned long long> binom((DIST_MAXU + 1) * (DIST_MAXR + 1));
    binom_table(binom.data());
    if (cudaMemcpyAsync(d->base + L.binom, binom.data(),
                        (size_t)L.brows * (DIST_MAXR + 1) * sizeof(unsigned long long),
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d->base + L.tables, p.tables.data(), p.tables.size() * sizeof(uint32_t),
                        cudaMemcpyHostToDevice, st) != cudaSuccess)
        return DIST_ECUDA;
    NoAllocExec ex{p, d, L, st};
    return solve_loop(p, ex, 0.0, out);
}
