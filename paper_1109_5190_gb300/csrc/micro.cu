// micro.cu -- project-written micro-benchmarks that give the rooflines'
// denominators: FP32 non-tensor FMA throughput (the walk is FP32 ALU work)
// and device copy bandwidth (the tree build is HBM streaming).
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
