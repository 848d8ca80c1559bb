// micro.cu -- project-written micro-benchmarks that give the rooflines'
// denominators: FP32 non-tensor FMA throughput (the walk's arithmetic is FP32
// ALU work), the L1 throughput of scattered 32-byte loads (the walk's node
// loads, one lane per particle, each lane at its own node) and device copy
// bandwidth (the tree build is HBM streaming).
#include <cmath>

#include "bh.h"
#include "bh_internal.cuh"

namespace bh {
namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;

// kChains independent FMA chains per thread keep every FP32 pipe busy;
// the result is stored so nothing is eliminated.
__global__ void __launch_bounds__(256) k_fma(float *out, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3f + c;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678f) out[blockIdx.x] = s;  // practically never true
}

constexpr int kGatherRecords = 2048;  // 64 KiB of 32-byte records: stays in every SM's L1
constexpr int kGatherIters = 4096;

// Every lane loads a pseudo-random 32-byte record (one 256-bit read-only load,
// like the walk's node load) from a table small enough to stay in L1, and
// keeps part of it so nothing is eliminated.  The indices come from a
// per-lane linear congruential sequence; four loads per step are independent.
__global__ void __launch_bounds__(512) k_l1_gather(const float4 *__restrict__ table, float *out)
{
    unsigned x = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 12345u;
    float acc = 0.f;
    for (int it = 0; it < kGatherIters; it += 4) {
        float v[4][8];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            x = x * 1664525u + 1013904223u;
            const float4 *p = table + 2 * ((x >> 16) & (kGatherRecords - 1));
            asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                         : "=f"(v[u][0]), "=f"(v[u][1]), "=f"(v[u][2]), "=f"(v[u][3]),
                           "=f"(v[u][4]), "=f"(v[u][5]), "=f"(v[u][6]), "=f"(v[u][7])
                         : "l"(p));
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) acc += v[u][0] + v[u][7];
    }
    if (acc == 12345.678f) out[blockIdx.x] = acc;  // practically never true
}

__global__ void __launch_bounds__(256) k_copy(const float4 *__restrict__ in, float4 *__restrict__ out,
                                             size_t n)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = in[i];
}

}  // namespace

double micro_fma_gflops(cudaStream_t st)
{
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    float *out = nullptr;
    if (cudaMalloc(&out, 4096 * sizeof(float)) != cudaSuccess) return -1.0;
    const int blocks = nsm * 8;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma<<<blocks, 256, 0, st>>>(out, 0.999999f, 1e-7f);  // warm-up
    double best = 0.0;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(e0, st);
        k_fma<<<blocks, 256, 0, st>>>(out, 0.999999f, 1e-7f);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double flops = 2.0 * kChains * kIters * (double)blocks * 256.0;
        const double g = flops / (ms * 1e-3) / 1e9;
        if (g > best) best = g;
    }
    g_launches += 6;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return best;
}

double micro_l1_sectors(cudaStream_t st)
{
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    float4 *table = nullptr;
    float *out = nullptr;
    if (cudaMalloc(&table, kGatherRecords * 32) != cudaSuccess) return -1.0;
    if (cudaMalloc(&out, 4096 * sizeof(float)) != cudaSuccess) { cudaFree(table); return -1.0; }
    cudaMemsetAsync(table, 0, kGatherRecords * 32, st);
    // the walk's configuration: the SM's storage given to L1, 48 warps per SM
    cudaFuncSetAttribute(k_l1_gather, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    const int blocks = nsm * 3;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_l1_gather<<<blocks, 512, 0, st>>>(table, out);  // warm-up
    // distinct sectors of one warp load: 32 lanes over kGatherRecords records
    const double r = kGatherRecords;
    const double per_request = r * (1.0 - std::pow(1.0 - 1.0 / r, 32.0));
    double best = 0.0;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(e0, st);
        k_l1_gather<<<blocks, 512, 0, st>>>(table, out);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double requests = (double)kGatherIters * blocks * (512 / 32);
        const double g = requests * per_request / (ms * 1e-3) / 1e9;
        if (g > best) best = g;
    }
    g_launches += 6;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(table);
    cudaFree(out);
    return best;
}

double micro_copy_gbs(size_t bytes, cudaStream_t st)
{
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const size_t n = bytes / 2 / sizeof(float4);
    float4 *a = nullptr, *b = nullptr;
    if (cudaMalloc(&a, n * sizeof(float4)) != cudaSuccess) return -1.0;
    if (cudaMalloc(&b, n * sizeof(float4)) != cudaSuccess) { cudaFree(a); return -1.0; }
    cudaMemsetAsync(a, 0, n * sizeof(float4), st);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = nsm * 8;
    k_copy<<<blocks, 256, 0, st>>>(a, b, n);
    double best = 0.0;
    for (int rep = 0; rep < 10; ++rep) {
        cudaEventRecord(e0, st);
        k_copy<<<blocks, 256, 0, st>>>(a, b, n);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double g = 2.0 * n * sizeof(float4) / (ms * 1e-3) / 1e9;
        if (g > best) best = g;
    }
    g_launches += 11;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(a);
    cudaFree(b);
    return best;
}

}  // namespace bh
