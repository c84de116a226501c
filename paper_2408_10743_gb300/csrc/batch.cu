// batch.cu -- step S7: many codes per launch, with continuous admission.
//
// A dist_batch owns one worker thread and one stream.  The worker runs
// "slices": it admits pending codes (up to a count and a device-footprint
// limit), plans the new ones, and packs the scratch set-ups and every active
// code's segments into one arena.  One replay of the slice graph uploads the
// arena, seeds the new codes' scratch, runs the multi-code launch
// (enum_batch_kernel) with a time budget and gathers every code's bound,
// counters and witness slot into one read-back; then, per code, the worker
// either certifies d, lets it resume in the next slice, or plans its next
// steps.  A code's chunk counter and bound stay
// on the device between slices, so a slice boundary loses no work.  Codes
// submitted while others are running join at the next slice: their work
// overlaps on the device with the codes already admitted.
//
// Certification after a slice (same argument as the single-code loop): with
// next = chunks claimed so far (every claimed chunk is finished before a
// launch ends), let s be the first planned step with U <= L_before(s).  If
// next has reached s's first chunk, every earlier step is complete and
// d = U.  If no such s exists and every chunk is done, the bound after the
// last planned step holds; d = U once it reaches U, otherwise the next
// steps are planned.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/dist.h"
#include "code.h"
#include "plan.h"
#include "pool.h"
#include "solve.h"

namespace dist {
cudaError_t slice_graph_build(unsigned char* d_arena, unsigned char* h_arena, const unsigned long long* binom,
                              int grid, int aux_grid, cudaEvent_t e0, cudaEvent_t e1, cudaStream_t st,
                              cudaGraph_t* graph, cudaGraphExec_t* exec, cudaGraphNode_t* h2d,
                              cudaGraphNode_t* d2h, cudaGraphNode_t* knode);
cudaError_t slice_graph_set_two(cudaGraphExec_t exec, cudaGraphNode_t knode, int two);
}  // namespace dist

using namespace dist;

namespace {

// A code with at most this many chunks is served entirely from the order list.
const unsigned long long kSmallChunks = 64;
// Host threads that plan, re-chunk and post-process a large slice.
// fn(a, b) over [0, n) on the process's host pool (this thread included),
// in ranges of `grain` items; every item is touched by exactly one thread.
template <class F>
void par_ranges(size_t n, size_t grain, const F& fn) {
    HostPool::get().run(n, grain, fn);
}

// Initial size of a batch's staging arena (pinned host and device): the
// slice of a few thousand small codes, with their tables, fits.
constexpr size_t kArenaInitialBytes = 32ull << 20;

struct Item {
    dist_code* c = nullptr;
    uint64_t ticket = 0;
    LaunchPlan lp;
    bool planned = false;
    int L = 0;                 // bound in force before lp's first step
    int r_next = 1, j_next = 0;
    int init_mode = 1;         // 1 = reset and seed, 2 = restart the counter, 0 = none
    int last_round = 0;
    int slices = 0;
    double work = 1.0;         // estimated_work of lp, set when it is planned
    bool done = false;
    dist_result res{};
    double t_submit = 0, t_admit = 0, t_done = 0;
    size_t footprint = 0;
};

struct Ticket {
    std::vector<Item*> items;
    int remaining = 0;
};

// Device buffer with a pinned host mirror; grows on demand.
template <class T>
struct DevBuf {
    T* d = nullptr;
    T* h = nullptr;
    size_t cap = 0;
    bool ensure(size_t n) {
        if (n <= cap) return true;
        size_t nc = std::max<size_t>(n, cap * 2 + 64);
        T *nd = nullptr, *nh = nullptr;
        if (cudaMalloc(&nd, nc * sizeof(T)) != cudaSuccess) return false;
        if (cudaMallocHost(&nh, nc * sizeof(T)) != cudaSuccess) {
            cudaFree(nd);
            return false;
        }
        release();
        d = nd;
        h = nh;
        cap = nc;
        return true;
    }
    void release() {
        if (d) cudaFree(d);
        if (h) cudaFreeHost(h);
        d = nullptr;
        h = nullptr;
        cap = 0;
    }
};

}  // namespace

struct dist_batch {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    int fatal = 0;
    dist_batch_opts opts{};
    DeviceCtx* dev = nullptr;
    cudaStream_t st = nullptr;
    std::deque<Item*> pending;
    std::vector<Item*> active;
    std::map<uint64_t, Ticket> tickets;
    std::deque<uint64_t> finished;    // tickets done and not yet reported by wait_any
    uint64_t next_ticket = 1;
    size_t resident = 0;
    // statistics
    uint64_t slices = 0;
    uint64_t launches = 0;
    uint64_t codes_done = 0;
    double gpu_seconds = 0;
    double plan_seconds = 0, post_seconds = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    // One slice's arena (SliceHeader, then its arrays), pinned on the host
    // and on the device, and the slice graph captured for this allocation.
    DevBuf<unsigned char> arena;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaGraphNode_t n_h2d = nullptr, n_d2h = nullptr, n_enum = nullptr;
    int graph_two = 0;  // the instance the graph's multi-code launch runs
    void drop_graph() {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        gexec = nullptr;
        graph = nullptr;
        graph_two = 0;
    }

    void run();
    int slice();
    void finish(Item* it, int status);
};

namespace {

// Estimated codewords of a plan: its steps whose L_before is below the
// random-code estimate of d (at least the first step).
double estimated_work(const Item* it) {
    const LaunchPlan& lp = it->lp;
    double w = 0;
    const int target = std::max(it->c->plan.d_est, lp.step_L_before.empty() ? 0 : lp.step_L_before[0] + 1);
    for (size_t s = 0; s < lp.step_r.size(); s++) {
        if (s > 0 && lp.step_L_before[s] >= target) break;
        const size_t e = s + 1 < lp.step_r.size() ? (size_t)lp.step_seg0[s + 1] : lp.segs.size();
        for (size_t k = (size_t)lp.step_seg0[s]; k < e; k++)
            w += (double)(lp.segs[k].rank1 - lp.segs[k].rank0) * (double)lp.segs[k].codes;
    }
    return std::max(w, 1.0);
}

}  // namespace

void dist_batch::finish(Item* it, int status) {
    it->done = true;
    it->t_done = wall_now();
    it->res.status = status;
    it->res.seconds = it->t_done - it->t_submit;
}

// One slice; returns a DIST_* error only for failures of the device itself.
int dist_batch::slice() {
    const double t_plan = wall_now();
    const int tw = dev->sms * dev->batch_blocks_per_sm * DIST_ENUM_WARPS;
    // plan codes that need it: first as if each had the whole GPU, then --
    // since the codes of a slice share the warps -- again with about four
    // times its share of the estimated work in warps, so that a small code is
    // cut into a few longer lane chunks instead of thousands of tiny ones
    std::vector<Item*> todo, fresh;
    for (Item* it : active)
        if (!it->planned && !it->done) todo.push_back(it);
    // plans are independent: large admissions are planned on several host
    // threads (each writes only its own items)
    std::vector<int> prc(todo.size(), P_OK);
    par_ranges(todo.size(), 32, [&](size_t a, size_t b) {
        for (size_t k = a; k < b; k++) {
            Item* it = todo[k];
            const Plan& p = it->c->plan;
            const int u0 = p.n_stab > 0 ? p.u0_excl : p.u0;
            prc[k] = plan_launch(p, it->r_next, it->j_next, it->L, u0, tw, 1e300, &it->lp);
            if (prc[k] == P_OK) it->work = estimated_work(it);  // re-chunking leaves it unchanged
        }
    });
    for (size_t k = 0; k < todo.size(); k++) {
        Item* it = todo[k];
        if (prc[k]) {
            finish(it, prc[k] == P_ERANGE ? DIST_ERANGE : DIST_EINVAL);
            continue;
        }
        it->planned = true;
        fresh.push_back(it);
    }
    // (only for run-to-completion launches: with a slice budget, short
    // chunks keep the slices short and the latency of new requests low)
    if (!fresh.empty() && opts.slice_ms <= 0) {
        double all = 0;
        for (Item* it : active)
            if (!it->done) all += it->work;
        par_ranges(fresh.size(), 32, [&](size_t a, size_t b) {
            for (size_t k = a; k < b; k++) {
                Item* it = fresh[k];
                const double share = it->work / std::max(all, 1.0);
                const int twi = (int)std::min<double>(tw, std::max(32.0, std::ceil(4.0 * share * tw)));
                if (twi < tw) plan_rechunk(&it->lp, twi);
            }
        });
    }
    std::vector<Item*> run;
    for (Item* it : active)
        if (!it->done) run.push_back(it);
    if (run.empty()) return DIST_OK;
    const int n = (int)run.size();
    // the slice's arrays, packed one after another into the arena behind
    // its header (offsets 256-byte aligned)
    size_t nseg = 0, ngam = 0, tab_bytes = 0;
    int ninit = 0;
    std::vector<Item*> inits_of;  // the items set up on the device in this slice
    for (Item* it : run) {
        nseg += it->lp.segs.size();
        ngam += it->lp.g.size();
        if (it->init_mode) {
            ninit++;
            inits_of.push_back(it);
            if (!it->c->tables_on_device) tab_bytes += (it->c->plan.tables.size() * 4 + 15) & ~(size_t)15;
        }
    }
    std::vector<double> work(n);
    double total = 0;
    for (int i = 0; i < n; i++) {
        work[i] = run[i]->work;
        total += work[i];
    }
    // Order list (phase 1, one chunk per entry), shortest job first so that
    // small -- typically newly admitted -- codes get warps at the start of
    // every slice.  A code with few chunks left gets one entry per chunk and
    // is done in phase 1; a large one gets entries in proportion to its share
    // of the work and goes into the ring that phase 2 probes.
    std::vector<int> idx(n);
    for (int i = 0; i < n; i++) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return work[a] < work[b]; });
    std::vector<int32_t> ord, rng;
    ord.reserve((size_t)n + tw);
    for (int i : idx) {
        const unsigned long long left = run[i]->lp.nchunks;  // upper bound on chunks still to claim
        if (left <= kSmallChunks) {
            for (unsigned long long k = 0; k < std::max(left, 1ull); k++) ord.push_back(i);
        } else {
            const long share = (long)floor(work[i] / total * (double)tw);
            for (long k = 0; k <= share; k++) ord.push_back(i);
        }
    }
    for (auto it = idx.rbegin(); it != idx.rend(); ++it)
        if (run[*it]->lp.nchunks > kSmallChunks) rng.push_back(*it);
    if (rng.empty()) rng.push_back(idx.back());
    SliceHeader hd;
    memset(&hd, 0, sizeof hd);
    size_t off = align256(sizeof(SliceHeader));
    auto place = [&](unsigned long long* o, size_t bytes) {
        *o = off;
        off = align256(off + bytes);
    };
    place(&hd.off_inits, (size_t)ninit * sizeof(BatchInit));
    place(&hd.off_codes, (size_t)n * sizeof(BatchCode));
    place(&hd.off_segs, nseg * sizeof(SegDesc));
    place(&hd.off_gammas, ngam * sizeof(GammaDesc));
    place(&hd.off_order, ord.size() * sizeof(int32_t));
    place(&hd.off_ring, rng.size() * sizeof(int32_t));
    place(&hd.off_sched, 2 * sizeof(unsigned long long));
    place(&hd.off_scrs, (size_t)n * sizeof(Scratch*));
    // tables of codes on their first slice (the init kernel copies them to
    // the codes' device blocks)
    unsigned long long off_tabs = 0;
    place(&off_tabs, tab_bytes);
    const size_t up_bytes = off;
    place(&hd.off_outs, (size_t)n * sizeof(BatchOut));
    if (off > arena.cap) {  // a new allocation: the graph is captured again
        drop_graph();
        if (!arena.ensure(off)) return DIST_ENOMEM;
    }
    unsigned char* const h = arena.h;
    hd.ncodes = n;
    hd.ninit = ninit;
    hd.norder = (int32_t)ord.size();
    hd.nring = (int32_t)rng.size();
    hd.budget_ns = opts.slice_ms > 0 ? (unsigned long long)(opts.slice_ms * 1e6) : 0ull;
    memcpy(h, &hd, sizeof hd);
    // scratch set-up of new and re-planned codes, with the tables of the
    // new ones (staged on the host threads)
    BatchInit* inits = reinterpret_cast<BatchInit*>(h + hd.off_inits);
    std::vector<unsigned long long> tab_at(inits_of.size(), 0);
    {
        unsigned long long o = off_tabs;
        for (size_t k = 0; k < inits_of.size(); k++) {
            const dist_code* c = inits_of[k]->c;
            if (c->tables_on_device) continue;
            tab_at[k] = o;
            o += (c->plan.tables.size() * 4 + 15) & ~(size_t)15;
        }
    }
    par_ranges(inits_of.size(), 64, [&](size_t a, size_t b) {
        for (size_t k = a; k < b; k++) {
            Item* it = inits_of[k];
            BatchInit& bi = inits[k];
            memset(&bi, 0, sizeof bi);
            bi.scr = it->c->d_scr;
            bi.mode = (uint32_t)it->init_mode;
            const Plan& p = it->c->plan;
            const int u0 = p.n_stab > 0 ? p.u0_excl : p.u0;
            bi.U0 = (uint32_t)std::min<int>(u0, DIST_WINF);
            bi.slot = p.n_stab > 0 ? p.u0_excl_slot : p.u0_slot;
            if (!it->c->tables_on_device) {
                bi.tab_dst = it->c->d_tables;
                bi.tab_off = tab_at[k];
                bi.tab_words = (uint32_t)p.tables.size();
                memcpy(h + tab_at[k], p.tables.data(), p.tables.size() * 4);
                it->c->tables_on_device = true;
            }
            it->init_mode = 0;
        }
    });
    BatchCode* codes = reinterpret_cast<BatchCode*>(h + hd.off_codes);
    SegDesc* segs = reinterpret_cast<SegDesc*>(h + hd.off_segs);
    GammaDesc* gammas = reinterpret_cast<GammaDesc*>(h + hd.off_gammas);
    Scratch** scrs = reinterpret_cast<Scratch**>(h + hd.off_scrs);
    // each code's segments and matrices at offsets fixed first, then packed
    // on the host threads
    std::vector<uint32_t> seg_at(n), gam_at(n);
    {
        size_t so = 0, go = 0;
        for (int i = 0; i < n; i++) {
            seg_at[i] = (uint32_t)so;
            gam_at[i] = (uint32_t)go;
            so += run[i]->lp.segs.size();
            go += run[i]->lp.g.size();
        }
    }
    par_ranges((size_t)n, 64, [&](size_t a, size_t b) {
        for (size_t i = a; i < b; i++) {
            Item* it = run[i];
            const Plan& p = it->c->plan;
            BatchCode& bc = codes[i];
            memset(&bc, 0, sizeof bc);
            bc.tables = it->c->d_tables;
            bc.scr = it->c->d_scr;
            for (int w = 0; w < DIST_MAXCW; w++) bc.outside[w] = p.outside[w];
            bc.W = p.W;
            bc.CW = p.CW;
            bc.proj = p.field == 4 ? 1 : 0;
            bc.exclude = p.n_stab > 0 ? 1 : 0;
            bc.seg0 = seg_at[i];
            bc.nseg = (uint32_t)it->lp.segs.size();
            bc.g0 = gam_at[i];
            bc.ng = (uint32_t)it->lp.g.size();
            bc.nchunks = it->lp.nchunks;
            memcpy(segs + seg_at[i], it->lp.segs.data(), it->lp.segs.size() * sizeof(SegDesc));
            memcpy(gammas + gam_at[i], it->lp.g.data(), it->lp.g.size() * sizeof(GammaDesc));
            scrs[i] = it->c->d_scr;
        }
    });
    memcpy(h + hd.off_order, ord.data(), ord.size() * sizeof(int32_t));
    memcpy(h + hd.off_ring, rng.data(), rng.size() * sizeof(int32_t));
    memset(h + hd.off_sched, 0, 2 * sizeof(unsigned long long));
    const int grid = dev->sms * dev->batch_blocks_per_sm;
    if (!gexec && slice_graph_build(arena.d, arena.h, dev->d_binom, grid, 2 * dev->sms, e0, e1, st, &graph,
                                    &gexec, &n_h2d, &n_d2h, &n_enum) != cudaSuccess)
        return DIST_ECUDA;
    // the two-word filter only where a code has three or more words per plane
    int two = 0;
    for (int i = 0; i < n && !two; i++) two = run[i]->c->plan.W >= 3 ? 1 : 0;
    if (two != graph_two) {
        if (slice_graph_set_two(gexec, n_enum, two) != cudaSuccess) return DIST_ECUDA;
        graph_two = two;
    }
    const double t_launch = wall_now();
    plan_seconds += t_launch - t_plan;
    // one upload, the slice graph, one read-back
    if (cudaGraphExecMemcpyNodeSetParams1D(gexec, n_h2d, arena.d, arena.h, up_bytes, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaGraphExecMemcpyNodeSetParams1D(gexec, n_d2h, arena.h + hd.off_outs, arena.d + hd.off_outs,
                                           (size_t)n * sizeof(BatchOut), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaGraphLaunch(gexec, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
        return DIST_ECUDA;
    const BatchOut* outs = reinterpret_cast<const BatchOut*>(arena.h + hd.off_outs);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    gpu_seconds += ms * 1e-3;
    launches++;
    slices++;
    // per code: certify, resume, or plan the next steps (each item is
    // touched by one host thread only)
    const double t_now = wall_now();
    par_ranges((size_t)n, 32, [&](size_t a, size_t b) {
    for (size_t i = a; i < b; i++) {
        Item* it = run[i];
        it->slices++;
        const BatchOut& o = outs[i];
        const LaunchPlan& lp = it->lp;
        const Plan& p = it->c->plan;
        const uint32_t U = o.U;
        const unsigned long long next = std::min(o.next_chunk, lp.nchunks);
        it->res.codewords = o.codewords;
        const SliceVerdict v = plan_after_slice(p, lp, U, next);
        it->last_round = std::max(it->last_round, v.last_round);
        if (v.kind != SLICE_CERTIFIED && opts.time_limit_s > 0 && t_now - it->t_admit > opts.time_limit_s) {
            // out of time: report the bounds reached, lower <= d <= U
            dist_result& r = it->res;
            r.k_eff = p.k_eff;
            r.n_gamma = (int)p.J.size();
            r.rounds = it->last_round;
            r.launches = (uint64_t)it->slices;
            r.lower = std::min<int>(plan_partial_bound(p, lp, next), (int)U);
            if (U != DIST_WINF) {
                r.d = (int)U;
                if (o.slot.claim == 0 || plan_decode(p, o.slot, r.witness, r.coeffs) != P_OK) {
                    finish(it, DIST_EINTERNAL);
                    continue;
                }
            }
            finish(it, DIST_EINCOMPLETE);
            continue;
        }
        if (v.kind == SLICE_REPLAN) {
            it->L = v.L;  // plan the following steps next slice
            it->r_next = lp.next_r;
            it->j_next = lp.next_jpos;
            it->planned = false;
            it->init_mode = 2;
        }
        const bool certified = v.kind == SLICE_CERTIFIED;
        if (!certified) continue;
        dist_result& r = it->res;
        r.k_eff = p.k_eff;
        r.n_gamma = (int)p.J.size();
        r.rounds = it->last_round;
        r.launches = (uint64_t)it->slices;
        if (U == DIST_WINF) {
            finish(it, DIST_EZERO);
            continue;
        }
        r.d = (int)U;
        r.lower = (int)U;
        if (o.slot.claim == 0 || plan_decode(p, o.slot, r.witness, r.coeffs) != P_OK) {
            finish(it, DIST_EINTERNAL);
            continue;
        }
        finish(it, DIST_OK);
    }
    });
    post_seconds += wall_now() - t_launch - ms * 1e-3;
    return DIST_OK;
}

void dist_batch::run() {
    cudaSetDevice(dev->device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        cv_work.wait(lk, [&] { return stop || !pending.empty() || !active.empty(); });
        if (stop) break;
        // admission by count and device footprint
        const size_t max_active = opts.max_active > 0 ? (size_t)opts.max_active : 8192;
        while (!pending.empty() && active.size() < max_active) {
            Item* it = pending.front();
            if (opts.max_resident_bytes && !active.empty() &&
                resident + it->footprint > opts.max_resident_bytes)
                break;
            pending.pop_front();
            it->t_admit = wall_now();
            resident += it->footprint;
            active.push_back(it);
        }
        lk.unlock();
        int rc = fatal ? fatal : slice();
        lk.lock();
        if (rc) {
            fatal = rc;
            for (Item* it : active)
                if (!it->done) finish(it, rc);
        }
        // retire finished codes and complete tickets
        std::vector<Item*> keep;
        for (Item* it : active) {
            if (!it->done) {
                keep.push_back(it);
                continue;
            }
            resident -= it->footprint;
            codes_done++;
            auto t = tickets.find(it->ticket);
            if (t != tickets.end() && --t->second.remaining == 0) finished.push_back(it->ticket);
        }
        active.swap(keep);
        cv_done.notify_all();
    }
}

extern "C" {

int dist_batch_create(dist_batch** out, const dist_batch_opts* opts) {
    if (!out) return DIST_EINVAL;
    *out = nullptr;
    DeviceCtx* dev = nullptr;
    int rc = device_ctx(&dev);
    if (rc) return rc;
    dist_batch* b = new (std::nothrow) dist_batch();
    if (!b) return DIST_ENOMEM;
    if (opts) b->opts = *opts;
    b->dev = dev;
    if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&b->e0) != cudaSuccess || cudaEventCreate(&b->e1) != cudaSuccess) {
        delete b;
        return DIST_ECUDA;
    }
    // the staging arena at its initial size and the slice graph on it, so
    // that the first slices allocate and capture nothing
    auto fail = [b](int rc) {
        b->drop_graph();
        b->arena.release();
        cudaEventDestroy(b->e0);
        cudaEventDestroy(b->e1);
        cudaStreamDestroy(b->st);
        delete b;
        return rc;
    };
    if (!b->arena.ensure(kArenaInitialBytes)) return fail(DIST_ENOMEM);
    if (slice_graph_build(b->arena.d, b->arena.h, dev->d_binom, dev->sms * dev->batch_blocks_per_sm, 2 * dev->sms,
                          b->e0, b->e1, b->st, &b->graph, &b->gexec, &b->n_h2d, &b->n_d2h, &b->n_enum) !=
        cudaSuccess)
        return fail(DIST_ECUDA);
    b->worker = std::thread([b] { b->run(); });
    *out = b;
    return DIST_OK;
}

int dist_batch_submit(dist_batch* b, dist_code* const* codes, int count, uint64_t* ticket) {
    if (!b || !codes || count < 1 || !ticket) return DIST_EINVAL;
    std::lock_guard<std::mutex> lk(b->mu);
    if (b->fatal) return b->fatal;
    for (int i = 0; i < count; i++) {
        if (!codes[i]) return DIST_EINVAL;
        if (codes[i]->in_batch || codes[i]->dev != b->dev) return DIST_EBUSY;
        if (codes[i]->plan.n_stab > 0 && codes[i]->plan.s_rank == codes[i]->plan.k_eff) return DIST_EZERO;
    }
    const double now = wall_now();
    const uint64_t id = b->next_ticket++;
    Ticket& t = b->tickets[id];
    for (int i = 0; i < count; i++) {
        Item* it = new Item();
        it->c = codes[i];
        it->c->in_batch = 1;
        it->ticket = id;
        it->t_submit = now;
        it->L = plan_initial_bound(it->c->plan);
        it->footprint = it->c->plan.tables.size() * 4 + sizeof(Scratch);
        t.items.push_back(it);
        b->pending.push_back(it);
    }
    t.remaining = count;
    *ticket = id;
    b->cv_work.notify_one();
    return DIST_OK;
}

static int collect(dist_batch* b, std::map<uint64_t, Ticket>::iterator t, dist_result* results) {
    for (auto f = b->finished.begin(); f != b->finished.end(); ++f)
        if (*f == t->first) {
            b->finished.erase(f);
            break;
        }
    for (size_t i = 0; i < t->second.items.size(); i++) {
        Item* it = t->second.items[i];
        if (results) results[i] = it->res;
        it->c->in_batch = 0;
        delete it;
    }
    b->tickets.erase(t);
    return DIST_OK;
}

int dist_batch_poll(dist_batch* b, uint64_t ticket, dist_result* results) {
    if (!b) return DIST_EINVAL;
    std::lock_guard<std::mutex> lk(b->mu);
    auto t = b->tickets.find(ticket);
    if (t == b->tickets.end()) return DIST_EINVAL;
    if (t->second.remaining > 0) return DIST_EBUSY;
    return collect(b, t, results);
}

int dist_batch_wait(dist_batch* b, uint64_t ticket, dist_result* results, double timeout_s) {
    if (!b) return DIST_EINVAL;
    std::unique_lock<std::mutex> lk(b->mu);
    auto t = b->tickets.find(ticket);
    if (t == b->tickets.end()) return DIST_EINVAL;
    auto ready = [&] { return t->second.remaining <= 0; };
    if (timeout_s > 0) {
        if (!b->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) return DIST_ETIMEOUT;
    } else {
        b->cv_done.wait(lk, ready);
    }
    return collect(b, t, results);
}

int dist_batch_wait_any(dist_batch* b, double timeout_s, uint64_t* ticket) {
    if (!b || !ticket) return DIST_EINVAL;
    std::unique_lock<std::mutex> lk(b->mu);
    auto ready = [&] { return !b->finished.empty() || b->fatal; };
    if (timeout_s > 0) {
        if (!b->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) return DIST_ETIMEOUT;
    } else {
        b->cv_done.wait(lk, ready);
    }
    if (b->finished.empty()) return b->fatal;
    *ticket = b->finished.front();
    b->finished.pop_front();
    return DIST_OK;
}

int dist_batch_stats(dist_batch* b, dist_batch_stats_t* s) {
    if (!b || !s) return DIST_EINVAL;
    std::lock_guard<std::mutex> lk(b->mu);
    memset(s, 0, sizeof *s);
    s->slices = b->slices;
    s->launches = b->launches;
    s->codes_done = b->codes_done;
    s->active = (uint64_t)b->active.size();
    s->pending = (uint64_t)b->pending.size();
    s->gpu_seconds = b->gpu_seconds;
    s->plan_seconds = b->plan_seconds;
    s->post_seconds = b->post_seconds;
    s->resident_bytes = (uint64_t)b->resident;
    return DIST_OK;
}

int dist_batch_destroy(dist_batch* b) {
    if (!b) return DIST_OK;
    {
        std::lock_guard<std::mutex> lk(b->mu);
        b->stop = true;
        b->cv_work.notify_all();
    }
    if (b->worker.joinable()) b->worker.join();
    cudaStreamSynchronize(b->st);
    for (auto& kv : b->tickets)
        for (Item* it : kv.second.items) {
            it->c->in_batch = 0;
            delete it;
        }
    b->drop_graph();
    b->arena.release();
    if (b->e0) cudaEventDestroy(b->e0);
    if (b->e1) cudaEventDestroy(b->e1);
    if (b->st) cudaStreamDestroy(b->st);
    delete b;
    return DIST_OK;
}

}  // extern "C"
