// api.cu -- the C ABI of libdist (declared in include/dist.h).
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <cmath>
#include <vector>

#include "../../include/dist.h"
#include "code.h"
#include "pool.h"
#include "plan.h"
#include "solve.h"

namespace dist {
cudaError_t enum_launch(const EnumParams& P, int grid, cudaStream_t st);
size_t enum_smem_bytes(const EnumParams& P);
int enum_blocks_per_sm(size_t smem);
size_t enum_max_dynamic_smem(size_t optin);
cudaError_t enum_set_max_smem(size_t bytes);
int batch_blocks_per_sm();
struct IntpeakRaw {
    double mix_s, popc_s, lop3_s;
    double sm_mhz;
    int sms, blocks, threads;
};
cudaError_t intpeak_run(int iters, cudaStream_t st, IntpeakRaw* r);
}  // namespace dist

using namespace dist;

namespace dist {

namespace {
std::mutex g_dev_mu;
DeviceCtx g_dev[64];
}  // namespace

// Copies a code's tables to the device if they are not there yet (a copy
// from pageable memory may return before its DMA lands, and the solves run
// on non-blocking streams, so it waits for the copy).
std::atomic<int> g_event_timing{0};

int upload_tables(dist_code* c) {
    if (c->tables_on_device) return DIST_OK;
    if (cudaMemcpy(c->d_tables, c->plan.tables.data(), c->plan.tables.size() * 4, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaStreamSynchronize(cudaStreamLegacy) != cudaSuccess)
        return DIST_ECUDA;
    c->tables_on_device = true;
    return DIST_OK;
}

int map_plan_rc(int rc) {
    switch (rc) {
        case P_OK: return DIST_OK;
        case P_EZERO: return DIST_EZERO;
        case P_ENOMEM: return DIST_ENOMEM;
        case P_ERANGE: return DIST_ERANGE;
        default: return DIST_EINVAL;
    }
}

int device_ctx(DeviceCtx** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return DIST_ECUDA;
    std::lock_guard<std::mutex> lk(g_dev_mu);
    DeviceCtx& d = g_dev[dev];
    if (d.device < 0) {
        int major = 0;
        if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess)
            return DIST_ECUDA;
        if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return DIST_ECUDA;
        std::vector<unsigned long long> tab((DIST_MAXU + 1) * (DIST_MAXR + 1));
        binom_table(tab.data());
        if (cudaMalloc(&d.d_binom, tab.size() * sizeof(unsigned long long)) != cudaSuccess)
            return DIST_ENOMEM;
        if (cudaMemcpy(d.d_binom, tab.data(), tab.size() * sizeof(unsigned long long),
                       cudaMemcpyHostToDevice) != cudaSuccess)
            return DIST_ECUDA;
        int optin = 0;
        if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            return DIST_ECUDA;
        d.smem_optin = enum_max_dynamic_smem((size_t)optin);
        if (d.smem_optin == 0 || enum_set_max_smem(d.smem_optin) != cudaSuccess) return DIST_ECUDA;
        d.blocks_per_sm = enum_blocks_per_sm(16 * 1024);
        d.batch_blocks_per_sm = batch_blocks_per_sm();
        if (d.blocks_per_sm < 1 || d.batch_blocks_per_sm < 1) return DIST_ECUDA;
        d.device = dev;
    }
    *out = &d;
    return DIST_OK;
}

namespace {
constexpr size_t kMaxIdleKits = 64;
constexpr size_t kMaxCachedBytes = 256ull << 20;
constexpr size_t kMinBlock = 32 * 1024;

void kit_destroy(SolveKit* k) {
    if (k->e0) cudaEventDestroy(k->e0);
    if (k->e1) cudaEventDestroy(k->e1);
    if (k->stream) cudaStreamDestroy(k->stream);
    if (k->h_state) cudaFreeHost(k->h_state);
    if (k->h_out) cudaFreeHost(k->h_out);
    delete k;
}
}  // namespace

int kit_acquire(DeviceCtx* d, SolveKit** out) {
    {
        std::lock_guard<std::mutex> lk(d->pool_mu);
        if (!d->kits.empty()) {
            *out = d->kits.back();
            d->kits.pop_back();
            return DIST_OK;
        }
    }
    SolveKit* k = new (std::nothrow) SolveKit();
    if (!k) return DIST_ENOMEM;
    if (cudaStreamCreateWithFlags(&k->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&k->e0) != cudaSuccess || cudaEventCreate(&k->e1) != cudaSuccess) {
        kit_destroy(k);
        return DIST_ECUDA;
    }
    if (cudaMallocHost(&k->h_state, state_bytes() + kKitTableBytes) != cudaSuccess) {
        k->h_state = nullptr;
        kit_destroy(k);
        return DIST_ENOMEM;
    }
    if (cudaHostAlloc(&k->h_out, sizeof(LaunchOut), cudaHostAllocMapped) != cudaSuccess) {
        k->h_out = nullptr;
        kit_destroy(k);
        return DIST_ENOMEM;
    }
    memset(k->h_out, 0, sizeof(LaunchOut));
    if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&k->d_out), k->h_out, 0) != cudaSuccess) {
        kit_destroy(k);
        return DIST_ECUDA;
    }
    *out = k;
    return DIST_OK;
}

void kit_release(DeviceCtx* d, SolveKit* k) {
    if (!k) return;
    {
        std::lock_guard<std::mutex> lk(d->pool_mu);
        if (d->kits.size() < kMaxIdleKits) {
            d->kits.push_back(k);
            return;
        }
    }
    kit_destroy(k);
}

int block_acquire(DeviceCtx* d, size_t bytes, void** out, size_t* cap) {
    size_t c = kMinBlock;
    while (c < bytes) c <<= 1;
    {
        std::lock_guard<std::mutex> lk(d->pool_mu);
        for (size_t i = 0; i < d->blocks.size(); i++)
            if (d->blocks[i].first == c) {
                *out = d->blocks[i].second;
                *cap = c;
                d->blocks[i] = d->blocks.back();
                d->blocks.pop_back();
                d->cached_bytes -= c;
                return DIST_OK;
            }
    }
    if (cudaMalloc(out, c) != cudaSuccess) {
        *out = nullptr;
        return DIST_ENOMEM;
    }
    *cap = c;
    return DIST_OK;
}

void block_release(DeviceCtx* d, void* p, size_t cap) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lk(d->pool_mu);
        if (d->cached_bytes + cap <= kMaxCachedBytes) {
            d->blocks.emplace_back(cap, p);
            d->cached_bytes += cap;
            return;
        }
    }
    cudaFree(p);
}

}  // namespace dist

namespace {

void release(dist_code* c) {
    if (!c) return;
    if (c->slab) {
        if (c->slab->refs.fetch_sub(1, std::memory_order_acq_rel) == 1) {
            cudaFree(c->slab->base);
            delete c->slab;
        }
    } else if (c->d_block) {
        block_release(c->dev, c->d_block, c->block_cap);
    }
    delete c;
}

// The device block's layout: tables, then scratch, then the segment table.
void place_block(dist_code* c, size_t tbytes) {
    c->d_tables = static_cast<uint32_t*>(c->d_block);
    c->d_scr = reinterpret_cast<Scratch*>(static_cast<unsigned char*>(c->d_block) + tbytes);
    c->d_segs = reinterpret_cast<SegDesc*>(reinterpret_cast<unsigned char*>(c->d_scr) + align256(sizeof(Scratch)));
}

// Runs one enumeration launch per call on the GPU (the executor of
// solve_loop).  The scratch (bound, counters, witness slots) is prepared on
// the host and goes to the device with the first launch's segment table in
// one copy; after every launch the kernel's last warp writes the bound, the
// counters and the witness slot of the bound to the kit's host-mapped
// LaunchOut, so nothing is copied back.
struct GpuExec {
    dist_code* c;
    SolveKit* kit;
    cudaStream_t st;
    double gpu_s = 0.0;
    unsigned long long nl = 0;
    bool first = true;  // the next launch uploads the scratch image too
    bool have_last = false;  // last_slot holds slot[last_U] after the last launch
    uint32_t last_U = DIST_WINF;
    WitnessSlot last_slot{};
    // kit staging: [table staging (kKitTableBytes) | scratch image | segment table]
    Scratch* hs() const { return reinterpret_cast<Scratch*>(kit->h_state + kKitTableBytes); }
    SegDesc* hsegs() const {
        return reinterpret_cast<SegDesc*>(kit->h_state + kKitTableBytes + align256(sizeof(Scratch)));
    }
    int reset() {
        memset(hs(), 0, sizeof(Scratch));
        hs()->U = DIST_WINF;
        first = true;
        have_last = false;
        return DIST_OK;
    }
    int seed(uint32_t U0, const WitnessSlot& s) {
        hs()->U = U0;
        hs()->slot[U0] = s;
        return DIST_OK;
    }
    int target_warps() const { return c->dev->sms * c->dev->blocks_per_sm * DIST_ENUM_WARPS; }
    double gpu_seconds() const { return gpu_s; }
    unsigned long long launches() const { return nl; }
    int run(const LaunchPlan& lp, double deadline_wall, StepResult* out) {
        EnumParams ep;
        plan_params(c->plan, lp, &ep);
        // U already at the random-code estimate of d: certification work
        ep.first_static = hs()->U <= (uint32_t)c->plan.d_est ? 1 : 0;
        ep.two_word = enum_two_word(ep, hs()->U);
        ep.tables = c->d_tables;
        ep.segs = c->d_segs;
        ep.binom = c->dev->d_binom;
        ep.scr = c->d_scr;
        ep.out = kit->d_out;
        ep.seq = ++kit->seq;
        ep.budget_ns = 0;
        if (deadline_wall > 0) {
            double left = deadline_wall - wall_now();
            ep.budget_ns = left > 1e-3 ? (unsigned long long)(left * 1e9) : 1000000ull;
        }
        const size_t smem = enum_smem_bytes(ep);
        if (smem > c->dev->smem_optin) return DIST_ERANGE;
        int bps = enum_blocks_per_sm(smem);
        if (bps < 1) return DIST_ECUDA;
        unsigned long long want = (lp.nchunks + DIST_ENUM_WARPS - 1) / DIST_ENUM_WARPS;
        if (want < 1) want = 1;
        const unsigned long long cap = (unsigned long long)c->dev->sms * (unsigned long long)bps;
        const int grid = (int)(want < cap ? want : cap);
        const size_t seg_bytes = lp.segs.size() * sizeof(SegDesc);
        memcpy(hsegs(), lp.segs.data(), seg_bytes);
        if (first) {
            // scratch image (next_chunk = 0) and segment table in one copy;
            // on the code's first solve its tables ride ahead of them, staged
            // so that the staging holds tables | scratch | segments at the
            // offsets the device block has them
            unsigned char* src = reinterpret_cast<unsigned char*>(hs());
            unsigned char* dst = reinterpret_cast<unsigned char*>(c->d_scr);
            size_t bytes = align256(sizeof(Scratch)) + seg_bytes;
            if (!c->tables_on_device) {  // at most kKitTableBytes (dist_init uploads larger ones)
                const size_t tb = align256(c->plan.tables.size() * 4);  // offset of d_scr in the block
                src -= tb;
                memcpy(src, c->plan.tables.data(), c->plan.tables.size() * 4);
                dst = static_cast<unsigned char*>(c->d_block);
                bytes += tb;
            }
            if (cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return DIST_ECUDA;
            c->tables_on_device = true;
            first = false;
        } else {
            if (cudaMemcpyAsync(c->d_segs, hsegs(), seg_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
                cudaMemsetAsync(&c->d_scr->next_chunk, 0, DIST_SCR_LAUNCH_RESET, st) != cudaSuccess)
                return DIST_ECUDA;
        }
        // CUDA events around the launch only when asked for: each timed
        // event adds about 11 us to a launch; the kernel stamps its own run
        // time either way
        const bool events = g_event_timing.load(std::memory_order_relaxed) != 0;
        if (events) cudaEventRecord(kit->e0, st);
        if (enum_launch(ep, grid, st) != cudaSuccess) return DIST_ECUDA;
        if (events) cudaEventRecord(kit->e1, st);
        nl++;
        if (cudaStreamSynchronize(st) != cudaSuccess) return DIST_ECUDA;
        const volatile LaunchOut* o = kit->h_out;
        if (o->seq != ep.seq) return DIST_EINTERNAL;  // the kernel always publishes
        hs()->U = o->U;
        hs()->status = o->status;
        hs()->codewords = o->codewords;
        last_U = o->U;
        memcpy(&last_slot, const_cast<const WitnessSlot*>(&o->slot), sizeof last_slot);
        have_last = true;
        if (events) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, kit->e0, kit->e1);
            gpu_s += ms * 1e-3;
        } else {
            gpu_s += stamps_seconds(o->t_first_inv, o->t_last);
        }
        out->U = hs()->U;
        out->status = hs()->status;
        out->codewords = hs()->codewords;
        return DIST_OK;
    }
    int read_slot(uint32_t w, WitnessSlot* s) {
        if (w > DIST_MAXN) return DIST_EINTERNAL;
        if (first) {  // no launch yet: the host image is the scratch
            *s = hs()->slot[w];
            return DIST_OK;
        }
        if (have_last && w == last_U) {  // published with the last launch
            *s = last_slot;
            return DIST_OK;
        }
        if (cudaMemcpyAsync(s, &c->d_scr->slot[w], sizeof *s, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return DIST_ECUDA;
        return DIST_OK;
    }
};

}  // namespace

extern "C" {

int dist_init(dist_code** out, const uint8_t* generator, int n, int K, int field) {
    if (!out || !generator) return DIST_EINVAL;
    *out = nullptr;
    dist_code* c = new (std::nothrow) dist_code();
    if (!c) return DIST_ENOMEM;
    int rc = map_plan_rc(plan_build(generator, n, K, field, &c->plan));
    if (rc) {
        delete c;
        return rc;
    }
    rc = device_ctx(&c->dev);
    if (rc) {
        delete c;
        return rc;
    }
    // One device block (from the per-device cache): tables, scratch, segment
    // table.  Streams, events and staging buffers come from the device's kit
    // cache at solve time (a code solved only in a batch never needs one).
    const size_t words = c->plan.tables.size();
    const size_t tbytes = align256(words * 4);
    rc = block_acquire(c->dev, tbytes + state_bytes(), &c->d_block, &c->block_cap);
    if (rc) {
        release(c);
        return rc;
    }
    place_block(c, tbytes);
    // Small tables go to the device with the first solve (one copy fewer
    // here); larger ones now.
    if (words * 4 > kKitTableBytes) {
        const int urc = upload_tables(c);
        if (urc) {
            release(c);
            return urc;
        }
    }
    *out = c;
    return DIST_OK;
}

int dist_init_many(dist_code** out, int count, const uint8_t* const* generators, const int* n, const int* K,
                   const int* field, int* status) {
    if (count < 0 || (count > 0 && (!out || !generators || !n || !K || !field || !status))) return DIST_EINVAL;
    for (int i = 0; i < count; i++) {
        out[i] = nullptr;
        status[i] = DIST_OK;
    }
    if (count == 0) return DIST_OK;
    DeviceCtx* dev = nullptr;
    int rc = device_ctx(&dev);
    if (rc) {
        for (int i = 0; i < count; i++) status[i] = rc;
        return rc;
    }
    // steps S1-S2 of every code on the host threads
    std::vector<dist_code*> cs((size_t)count, nullptr);
    HostPool::get().run((size_t)count, 4, [&](size_t a, size_t b) {
        for (size_t i = a; i < b; i++) {
            if (!generators[i]) {
                status[i] = DIST_EINVAL;
                continue;
            }
            dist_code* c = new (std::nothrow) dist_code();
            if (!c) {
                status[i] = DIST_ENOMEM;
                continue;
            }
            const int prc = map_plan_rc(plan_build(generators[i], n[i], K[i], field[i], &c->plan));
            if (prc) {
                delete c;
                status[i] = prc;
                continue;
            }
            cs[i] = c;
        }
    });
    // one device allocation for all of them: each code's block holds its
    // tables, scratch and segment table, 256-byte aligned
    std::vector<size_t> off((size_t)count, 0);
    size_t total = 0;
    int live = 0;
    for (int i = 0; i < count; i++) {
        if (!cs[i]) continue;
        off[i] = total;
        total += align256(align256(cs[i]->plan.tables.size() * 4) + state_bytes());
        live++;
    }
    DevSlab* slab = nullptr;
    if (live > 0) {
        slab = new (std::nothrow) DevSlab();
        if (!slab || cudaMalloc(&slab->base, total) != cudaSuccess) {
            delete slab;
            for (int i = 0; i < count; i++)
                if (cs[i]) {
                    delete cs[i];
                    cs[i] = nullptr;
                    status[i] = DIST_ENOMEM;
                }
            slab = nullptr;
        } else {
            slab->refs.store(live);
        }
    }
    int first_err = DIST_OK;
    for (int i = 0; i < count; i++) {
        dist_code* c = cs[i];
        if (c) {
            const size_t tbytes = align256(c->plan.tables.size() * 4);
            c->dev = dev;
            c->slab = slab;
            c->d_block = static_cast<unsigned char*>(slab->base) + off[i];
            c->block_cap = align256(tbytes + state_bytes());
            place_block(c, tbytes);
            if (c->plan.tables.size() * 4 > kKitTableBytes) {  // as dist_init: larger tables now
                const int urc = upload_tables(c);
                if (urc) {
                    release(c);
                    c = nullptr;
                    status[i] = urc;
                }
            }
            out[i] = c;
        }
        if (status[i] && first_err == DIST_OK) first_err = status[i];
    }
    return first_err;
}

int dist_normalizer(const uint8_t* stabilizers, int n, int m, uint8_t* generator_out, int* K_out,
                    int* n_stab_out) {
    if (!stabilizers || !generator_out || !K_out || !n_stab_out) return DIST_EINVAL;
    std::vector<uint8_t> gen;
    int K = 0, s = 0;
    const int rc = map_plan_rc(stab_normalizer(stabilizers, n, m, &gen, &K, &s));
    if (rc) return rc;
    memcpy(generator_out, gen.data(), gen.size());
    *K_out = K;
    *n_stab_out = s;
    return DIST_OK;
}

int dist_init_stabilizer(dist_code** out, const uint8_t* stabilizers, int n, int m) {
    if (!out || !stabilizers) return DIST_EINVAL;
    *out = nullptr;
    std::vector<uint8_t> gen;
    int K = 0, s = 0;
    int rc = map_plan_rc(stab_normalizer(stabilizers, n, m, &gen, &K, &s));
    if (rc) return rc;
    rc = dist_init(out, gen.data(), n, K, DIST_F2);
    if (rc) return rc;
    if (s > 0) {
        rc = dist_set_exclude(*out, s);
        if (rc) {
            dist_free(*out);
            *out = nullptr;
            return rc;
        }
    }
    return DIST_OK;
}

int dist_set_exclude(dist_code* c, int n_stab) {
    if (!c) return DIST_EINVAL;
    return map_plan_rc(plan_set_exclude(&c->plan, n_stab));
}

int dist_solve_bounded(dist_code* c, dist_result* out, void* cuda_stream, double time_limit_s) {
    if (!c || !out) return DIST_EINVAL;
    if (c->in_batch) return DIST_EBUSY;
    if (c->plan.n_stab > 0 && c->plan.s_rank == c->plan.k_eff) return DIST_EZERO;
    DeviceGuard guard(c->dev->device);
    SolveKit* kit = nullptr;
    int rc = kit_acquire(c->dev, &kit);
    if (rc) return rc;
    GpuExec ex{c, kit, cuda_stream ? (cudaStream_t)cuda_stream : kit->stream};
    rc = solve_loop(c->plan, ex, time_limit_s, out);
    // every launch of the solve was synchronized; on an error path, drain the
    // stream before the kit's staging buffer can serve another solve
    if (rc != DIST_OK && rc != DIST_EINCOMPLETE && rc != DIST_EZERO) cudaStreamSynchronize(ex.st);
    kit_release(c->dev, kit);
    return rc;
}

int dist_solve(dist_code* c, dist_result* out, void* cuda_stream) {
    return dist_solve_bounded(c, out, cuda_stream, 0.0);
}

int dist_free(dist_code* c) {
    if (!c) return DIST_OK;
    if (c->in_batch) return DIST_EBUSY;
    DeviceGuard guard(c->dev ? c->dev->device : 0);
    release(c);
    return DIST_OK;
}

int dist_plan_info_get(const uint8_t* generator, int n, int K, int field, int n_stab,
                       dist_plan_info* info) {
    if (!info) return DIST_EINVAL;
    memset(info, 0, sizeof *info);
    Plan p;
    int rc = map_plan_rc(plan_build(generator, n, K, field, &p));
    if (rc) return rc;
    if (n_stab) {
        rc = map_plan_rc(plan_set_exclude(&p, n_stab));
        if (rc) return rc;
    }
    info->n_gamma_built = (int)p.gammas.size();
    info->n_gamma_used = (int)p.J.size();
    info->k_eff = p.k_eff;
    info->s_rank = p.s_rank;
    info->d_est = p.d_est;
    info->u0 = p.u0;
    for (size_t t = 0; t < p.J.size() && t < 16; t++) info->order[t] = p.J[t];
    for (size_t g = 0; g < p.gammas.size() && g < 16; g++) {
        info->a[g] = (int)p.gammas[g].A.size();
        info->b[g] = (int)p.gammas[g].B.size();
        info->f[g] = p.gammas[g].f;
    }
    return DIST_OK;
}

int dist_plan_unit(const uint8_t* generator, int n, int K, int field, int gamma, int unit, int rep,
                   uint8_t* vec_out, int* qubit, int* kind) {
    if (!vec_out) return DIST_EINVAL;
    Plan p;
    int rc = map_plan_rc(plan_build(generator, n, K, field, &p));
    if (rc) return rc;
    if (gamma < 0 || gamma >= (int)p.gammas.size()) return DIST_EINVAL;
    const Gamma& G = p.gammas[gamma];
    if (unit < 0 || unit >= G.units()) return DIST_EINVAL;
    const Unit& x = unit < (int)G.A.size() ? G.A[unit] : G.B[unit - G.A.size()];
    if (rep < 0 || rep >= x.nrep) return DIST_EINVAL;
    for (int i = 0; i < n; i++) {
        vec_out[i] = (uint8_t)((x.rep[rep].x[i >> 5] >> (i & 31)) & 1u);
        vec_out[n + i] = (uint8_t)((x.rep[rep].z[i >> 5] >> (i & 31)) & 1u);
    }
    if (qubit) *qubit = x.qubit;
    if (kind) *kind = x.kind;
    return DIST_OK;
}

int dist_intpeak(dist_intpeak_result* out, int iters, void* cuda_stream) {
    if (!out || iters < 1) return DIST_EINVAL;
    memset(out, 0, sizeof *out);
    IntpeakRaw r;
    if (intpeak_run(iters, (cudaStream_t)cuda_stream, &r) != cudaSuccess) return DIST_ECUDA;
    const double threads = (double)r.blocks * r.threads;
    out->mix_per_s = threads * (double)iters * 81.0 / r.mix_s;
    out->popc_per_s = threads * (double)iters * 8.0 / r.popc_s;
    out->lop3_per_s = threads * (double)iters * 8.0 / r.lop3_s;
    out->sm_mhz = r.sm_mhz;
    out->sms = r.sms;
    out->blocks = r.blocks;
    return DIST_OK;
}

int dist_set_tuning(const dist_tuning* t) {
    if (!t) return DIST_EINVAL;
    Tuning cur = tuning_get();
    if (t->chunks_per_warp > 0) cur.chunks_per_warp = t->chunks_per_warp;
    if (t->lane_cap_log2 > 0) cur.lane_cap_log2 = t->lane_cap_log2;
    if (t->lane_floor_log2 > 0) cur.lane_floor_log2 = t->lane_floor_log2;
    tuning_set(cur);
    return DIST_OK;
}

int dist_set_plan_search(int trials) {
    if (trials < 0) return DIST_EINVAL;
    plan_set_search_trials(trials);
    return DIST_OK;
}

int dist_get_plan_search(void) { return plan_search_trials(); }

int dist_set_gamma_limit(int m) {
    if (m < 0) return DIST_EINVAL;
    plan_set_gamma_limit(m);
    return DIST_OK;
}

int dist_get_gamma_limit(void) { return plan_gamma_limit(); }

int dist_set_event_timing(int on) {
    g_event_timing.store(on ? 1 : 0);
    return DIST_OK;
}

int dist_get_event_timing(void) { return g_event_timing.load(); }

int dist_get_tuning(dist_tuning* t) {
    if (!t) return DIST_EINVAL;
    const Tuning cur = tuning_get();
    t->chunks_per_warp = cur.chunks_per_warp;
    t->lane_cap_log2 = cur.lane_cap_log2;
    t->lane_floor_log2 = cur.lane_floor_log2;
    t->codewords_per_s = 0.0;
    return DIST_OK;
}

// Calibration: two seeded random codes (n = 64, K = 56 and n = 72, K = 72)
// whose solves are dominated by one large enumeration step, timed with the
// kernels' CUDA events for each setting of the grid; best median rate wins.
namespace {

// Digest of the launches a solve of c would make under the tuning in force
// if U stayed at its seed: the round loop's plan_launch sequence, segment
// tables and chunk counts.  Two settings with the same digest cut every
// launch the same way (U only decides where a solve stops), so only one of
// them needs timing.
unsigned long long launch_sequence_digest(const dist_code* c) {
    const Plan& p = c->plan;
    unsigned long long h = 1469598103934665603ull;
    auto put = [&h](const void* d, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(d);
        for (size_t i = 0; i < n; i++) h = (h ^ b[i]) * 1099511628211ull;
    };
    const int ub = seed_bound(p);
    const int warps = c->dev->sms * c->dev->blocks_per_sm * DIST_ENUM_WARPS;
    int r = 1, jpos = 0, L = plan_initial_bound(p);
    for (int launch = 0; launch < 64; launch++) {
        LaunchPlan lp;
        const int rc = plan_launch(p, r, jpos, L, ub, warps, kLaunchCodewords, &lp);
        put(&rc, sizeof rc);
        if (rc) break;
        put(&lp.nchunks, sizeof lp.nchunks);
        for (const SegDesc& sg : lp.segs) put(&sg, sizeof sg);
        L = plan_lower_bound(p, lp.step_r.back(), lp.step_jpos.back());
        if (L == (int)DIST_WINF || (ub < (int)DIST_WINF && L >= ub)) break;
        r = lp.next_r;
        jpos = lp.next_jpos;
    }
    return h;
}

// Times two solves of every code per setting of the grid (the second one
// counts) and applies the setting with the best geometric-mean codewords/s,
// the setting in force winning unless another is 2 % faster.  A setting
// whose launches are those of a setting already timed is not timed again.
int autotune_on(const std::vector<dist_code*>& codes, double budget_s, dist_tuning* best) {
    const Tuning saved = tuning_get();
    // the setting in force is timed first and kept unless another one is
    // at least 2 % faster: on codes whose launches the tuning does not
    // reach, the choice would otherwise follow timing noise
    std::vector<Tuning> grid{saved};
    for (int a : {2, 3, 6, 12})
        for (int b : {13, 14, 16})
            for (int f : {8, 10, 12}) {
                Tuning t;
                t.chunks_per_warp = a;
                t.lane_cap_log2 = b;
                t.lane_floor_log2 = f;
                grid.push_back(t);
            }
    double best_rate = -1;
    Tuning best_t = saved;
    const double t0 = wall_now();
    std::vector<std::vector<unsigned long long>> seen;
    for (const Tuning& t : grid) {
        if (wall_now() - t0 > budget_s) break;
        tuning_set(t);
        std::vector<unsigned long long> sig;
        for (dist_code* c : codes) sig.push_back(launch_sequence_digest(c));
        if (std::find(seen.begin(), seen.end(), sig) != seen.end()) continue;
        seen.push_back(sig);
        // geometric mean of the per-code rates: a short solve weighs as much
        // as a long one
        double log_rate = 0;
        for (dist_code* c : codes) {
            dist_result r;
            for (int rep = 0; rep < 2; rep++) {
                int rc = dist_solve(c, &r, nullptr);
                if (rc != DIST_OK) {
                    tuning_set(saved);
                    return rc;
                }
                if (rep == 1) log_rate += std::log((double)r.codewords / std::max(r.gpu_seconds, 1e-9));
            }
        }
        const double rate = std::exp(log_rate / (double)codes.size());
        if (best_rate < 0 || rate > 1.02 * best_rate) {
            best_rate = rate;
            best_t = t;
        }
    }
    tuning_set(best_t);
    best->chunks_per_warp = best_t.chunks_per_warp;
    best->lane_cap_log2 = best_t.lane_cap_log2;
    best->lane_floor_log2 = best_t.lane_floor_log2;
    best->codewords_per_s = best_rate;
    return DIST_OK;
}

}  // namespace

int dist_autotune(dist_tuning* best, double budget_s) {
    if (!best) return DIST_EINVAL;
    if (budget_s <= 0) budget_s = 10.0;
    static const int kSizes[2][2] = {{64, 56}, {72, 72}};
    std::vector<dist_code*> codes;
    uint64_t x = 0x9E3779B97F4A7C15ull;  // xorshift64* stream for the calibration bits
    for (auto& nk : kSizes) {
        const int n = nk[0], K = nk[1];
        for (int attempt = 0; attempt < 100; attempt++) {
            std::vector<uint8_t> g((size_t)K * 2 * n);
            for (auto& b : g) {
                x ^= x >> 12;
                x ^= x << 25;
                x ^= x >> 27;
                b = (uint8_t)(((x * 0x2545F4914F6CDD1Dull) >> 63) & 1u);
            }
            dist_code* c = nullptr;
            int rc = dist_init(&c, g.data(), n, K, DIST_F2);
            if (rc == DIST_OK && c->plan.k_eff == K) {
                codes.push_back(c);
                break;
            }
            if (c) dist_free(c);
            if (rc != DIST_OK && rc != DIST_EZERO) {
                for (dist_code* cc : codes) dist_free(cc);
                return rc;
            }
        }
    }
    const int rc = autotune_on(codes, budget_s, best);
    for (dist_code* c : codes) dist_free(c);
    return rc;
}

int dist_autotune_codes(dist_code* const* codes, int count, double budget_s, dist_tuning* best) {
    if (!best || !codes || count < 1) return DIST_EINVAL;
    if (budget_s <= 0) budget_s = 10.0;
    std::vector<dist_code*> v;
    for (int i = 0; i < count; i++) {
        if (!codes[i]) return DIST_EINVAL;
        if (codes[i]->in_batch) return DIST_EBUSY;
        v.push_back(codes[i]);
    }
    return autotune_on(v, budget_s, best);
}

const char* dist_version(void) { return "libdist 0.1 (sm_103a)"; }

const char* dist_strerror(int code) {
    switch (code) {
        case DIST_OK: return "ok";
        case DIST_EINVAL: return "invalid argument";
        case DIST_ENOMEM: return "out of memory";
        case DIST_ECUDA: return "CUDA error or no usable device";
        case DIST_ETIMEOUT: return "bounded wait timed out";
        case DIST_EINCOMPLETE: return "time limit reached before d was certified";
        case DIST_EZERO: return "no nonzero codeword (outside the excluded span)";
        case DIST_EBUSY: return "not finished yet";
        case DIST_EINTERNAL: return "internal self-check failed";
        case DIST_ERANGE: return "distance needs combinations beyond the device walk";
        default: return "unknown error";
    }
}

}  // extern "C"
