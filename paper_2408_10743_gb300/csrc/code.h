// code.h -- library-internal definitions shared by the C-ABI translation units.
#pragma once
#include <cuda_runtime.h>

#include "plan.h"

namespace dist {

// Per-device constants: the binomial table the kernels unrank with, SM count
// and occupancy.
struct DeviceCtx {
    int device = -1;
    int sms = 0;
    int blocks_per_sm = 0;          // single-code kernel at a small shared-memory footprint
    int batch_blocks_per_sm = 0;    // multi-code kernel
    size_t smem_optin = 0;          // largest dynamic shared memory per block
    unsigned long long* d_binom = nullptr;
};

// Context of the current device (created on first use).
int device_ctx(DeviceCtx** out);

int map_plan_rc(int rc);

}  // namespace dist

// A code resident on one device: its plan, its tables and its scratch.
struct dist_code {
    dist::Plan plan;
    dist::DeviceCtx* dev = nullptr;
    uint32_t* d_tables = nullptr;             // Plan::tables on the device
    SegDesc* d_segs = nullptr;          // segment table of the current launch
    SegDesc* h_segs = nullptr;          // pinned staging copy
    Scratch* d_scr = nullptr;           // bound, counters, witness slots
    Scratch* h_scr = nullptr;           // pinned mirror for read-back
    cudaStream_t stream = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int in_batch = 0;                         // owned by a batch ticket until it completes
};
