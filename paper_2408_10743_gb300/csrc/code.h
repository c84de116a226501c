// code.h -- library-internal definitions shared by the C-ABI translation units.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <utility>
#include <vector>

#include "plan.h"

namespace dist {

// What one single-code solve needs besides the code's own device block: a
// stream (used when the caller passes none), timing events, and a pinned
// staging area holding a Scratch image followed by a segment table, laid out
// like the device block's tail so that one copy moves both.
struct SolveKit {
    cudaStream_t stream = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    unsigned char* h_state = nullptr;
    LaunchOut* h_out = nullptr;     // host-mapped launch result (LaunchOut)
    LaunchOut* d_out = nullptr;     // its device address
    unsigned long long seq = 0;     // launches made with this kit
};

// Per-device constants (the binomial table the kernels unrank with, SM count,
// occupancy) and caches of solve kits and device blocks, so that dist_init,
// dist_solve and dist_free make no CUDA allocation once warm.
struct DeviceCtx {
    int device = -1;
    int sms = 0;
    int blocks_per_sm = 0;          // single-code kernel at a small shared-memory footprint
    int batch_blocks_per_sm = 0;    // multi-code kernel
    size_t smem_optin = 0;          // largest dynamic shared memory per enumeration block
    unsigned long long* d_binom = nullptr;
    std::mutex pool_mu;
    std::vector<SolveKit*> kits;                     // idle kits
    std::vector<std::pair<size_t, void*>> blocks;    // idle device blocks (capacity, pointer)
    size_t cached_bytes = 0;                         // capacity held in `blocks`
};

// Context of the current device (created on first use).
int device_ctx(DeviceCtx** out);

// Kit for one solve: an idle one, else a new one; back to the cache after.
int kit_acquire(DeviceCtx* d, SolveKit** out);
void kit_release(DeviceCtx* d, SolveKit* k);

// Device block of at least `bytes` (power-of-two capacity, at least 32 KB)
// from the cache, else cudaMalloc; a released block stays cached while the
// cache holds less than 256 MB.
int block_acquire(DeviceCtx* d, size_t bytes, void** out, size_t* cap);
void block_release(DeviceCtx* d, void* p, size_t cap);

// Byte layout of a code's device block: tables, then Scratch, then the
// segment table of the current single-code launch.
inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
inline size_t state_bytes() { return align256(sizeof(Scratch)) + DIST_MAXSEG * sizeof(SegDesc); }
// Tables of at most this many bytes go to the device with a code's first
// solve, staged in the solve kit behind its scratch image, instead of by a
// separate synchronous copy in dist_init.
constexpr size_t kKitTableBytes = 64 * 1024;

int map_plan_rc(int rc);
// Per-launch CUDA-event timing of single-code solves (dist_set_event_timing).
extern std::atomic<int> g_event_timing;
// Copies c's tables to the device unless they are there already (synchronous).
int upload_tables(dist_code* c);

// Makes a device current for a scope and restores the previous one.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace dist

// A code resident on one device: its plan and one device block holding its
// tables, its scratch and its launch segment table.
namespace dist {
// One device allocation shared by the codes of a dist_init_many call; freed
// when the last of them is.
struct DevSlab {
    void* base = nullptr;
    std::atomic<int> refs{0};
};
}  // namespace dist

struct dist_code {
    dist::Plan plan;
    dist::DeviceCtx* dev = nullptr;
    void* d_block = nullptr;
    size_t block_cap = 0;
    dist::DevSlab* slab = nullptr;            // d_block lies in a shared allocation (dist_init_many)
    uint32_t* d_tables = nullptr;             // Plan::tables on the device
    Scratch* d_scr = nullptr;                 // bound, counters, witness slots
    SegDesc* d_segs = nullptr;                // segment table of the current launch (after d_scr)
    bool tables_on_device = false;            // Plan::tables copied to d_tables
    int in_batch = 0;                         // owned by a batch ticket until it completes
};
