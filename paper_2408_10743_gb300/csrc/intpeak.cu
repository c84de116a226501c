// intpeak.cu -- integer-issue microbenchmark: the roofline denominator of the
// enumeration kernel, measured on the device it runs on.
//
//  * mix:  the enumeration's inner block exactly -- a 9-entry register table
//          swept 9 times with 8 base steps in between (81 codewords); per
//          codeword t = (bx ^ Tx) | (bz ^ Tz), c = popc(t), folded with 3-way
//          mins (two LOP3, one POPC, half a min).  Result: codewords per second
//          the instruction mix allows.
//  * popc: eight independent chains of popc(a ^ k).
//  * lop3: eight independent chains of three-input logic ops.
// Every kernel stores a data-dependent value so nothing is dead code.
#include <cuda_runtime.h>
#include <stdint.h>

namespace dist {

__device__ __forceinline__ unsigned long long ip_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void __launch_bounds__(256, 2) intpeak_mix(int iters, const uint32_t* seed, uint32_t* out,
                                                    unsigned long long* clk) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t Tx[9], Tz[9], D[6];
#pragma unroll
    for (int j = 0; j < 9; j++) {  // loaded, so the compiler cannot fold them into immediates
        Tx[j] = seed[(tid + 2 * j) & 1023];
        Tz[j] = seed[(tid + 2 * j + 1) & 1023];
    }
#pragma unroll
    for (int j = 0; j < 6; j++) D[j] = seed[(tid + 31 * j + 7) & 1023];
    uint32_t bx = tid, bz = ~tid, acc = 0;
    unsigned long long c0 = 0, g0 = 0;
    if (tid == 0) {
        c0 = clock64();
        g0 = ip_ns();
    }
    for (int it = 0; it < iters; it++) {
        uint32_t m = 0xFFFFu;
#pragma unroll
        for (int s = 0; s < 9; s++) {  // 9 sweeps of 9 codewords, 8 base steps: 81 codewords
            uint32_t c[9];
#pragma unroll
            for (int j = 0; j < 9; j++) c[j] = (uint32_t)__popc((bx ^ Tx[j]) | (bz ^ Tz[j]));
            m = __vimin3_u32(m, __vimin3_u32(c[0], c[1], c[2]), __vimin3_u32(c[3], c[4], c[5]));
            m = __vimin3_u32(m, __vimin3_u32(c[6], c[7], c[8]), m);
            if (s < 8) {
                bx ^= D[s % 3];
                bz ^= D[3 + s % 3];
            }
        }
        acc += m;
        bx += 0x9E3779B9u;
    }
    if (tid == 0) {
        clk[0] = clock64() - c0;
        clk[1] = ip_ns() - g0;
    }
    if (acc == 0x7FFFFFFFu) out[tid] = acc;
}

__global__ void __launch_bounds__(256) intpeak_popc(int iters, uint32_t* out) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t a[8];
#pragma unroll
    for (int k = 0; k < 8; k++) a[k] = tid * (2u * k + 1u);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < 8; k++) a[k] = (uint32_t)__popc(a[k] ^ (0x5A5A5A5Au + 0x01010101u * k + it));
    }
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) s += a[k];
    if (s == 0xFFFFFFFFu) out[tid] = s;
}

__global__ void __launch_bounds__(256) intpeak_lop3(int iters, uint32_t* out) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t a[8];
#pragma unroll
    for (int k = 0; k < 8; k++) a[k] = tid * (2u * k + 1u) + k;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < 8; k++) a[k] = (a[k] ^ a[(k + 1) & 7]) | (a[(k + 3) & 7] & ~a[(k + 5) & 7]);
    }
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) s ^= a[k];
    if (s == 0x12345678u) out[tid] = s;
}

struct IntpeakRaw {
    double mix_s, popc_s, lop3_s;
    double sm_mhz;
    int sms, blocks, threads;
};

cudaError_t intpeak_run(int iters, cudaStream_t st, IntpeakRaw* r) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return e;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, intpeak_mix, 256, 0);
    if (nb < 1) nb = 1;
    const int blocks = sms * nb;
    uint32_t* out = nullptr;
    uint32_t* seed = nullptr;
    unsigned long long* clk = nullptr;
    if ((e = cudaMalloc(&out, (size_t)blocks * 256 * 4))) return e;
    if ((e = cudaMalloc(&clk, 16)) || (e = cudaMalloc(&seed, 1024 * 4))) {
        cudaFree(out);
        if (clk) cudaFree(clk);
        return e;
    }
    {
        uint32_t h[1024];
        uint32_t x = 0x12345679u;
        for (int i = 0; i < 1024; i++) {  // xorshift32
            x ^= x << 13;
            x ^= x >> 17;
            x ^= x << 5;
            h[i] = x;
        }
        cudaMemcpy(seed, h, sizeof h, cudaMemcpyHostToDevice);
    }
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float ms = 0;
    // warm-up
    intpeak_mix<<<blocks, 256, 0, st>>>(iters / 8 + 1, seed, out, clk);
    cudaEventRecord(a, st);
    intpeak_mix<<<blocks, 256, 0, st>>>(iters, seed, out, clk);
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
    r->mix_s = ms * 1e-3;
    unsigned long long hclk[2] = {0, 0};
    cudaMemcpy(hclk, clk, 16, cudaMemcpyDeviceToHost);
    r->sm_mhz = hclk[1] ? (double)hclk[0] / (double)hclk[1] * 1e3 : 0.0;
    cudaEventRecord(a, st);
    intpeak_popc<<<blocks, 256, 0, st>>>(iters, out);
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
    r->popc_s = ms * 1e-3;
    cudaEventRecord(a, st);
    intpeak_lop3<<<blocks, 256, 0, st>>>(iters, out);
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
    r->lop3_s = ms * 1e-3;
    e = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    cudaFree(clk);
    cudaFree(seed);
    r->sms = sms;
    r->blocks = blocks;
    r->threads = 256;
    return e;
}

}  // namespace dist
