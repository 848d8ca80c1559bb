// noalloc.cu -- Morton keys of one system without any device allocation.
//
// Who this is for: code that cannot call cudaMalloc.  cudaMalloc may block
// until the whole device is idle and can fail when another allocator (a
// framework's caching allocator, a pre-carved memory pool) already holds the
// free memory; a caller on a latency-critical loop, or one that owns no
// allocator at all, can still compute keys here.  The caller passes the
// inputs and outputs; the only scratch the kernels need -- per-chunk bounding
// boxes and the derived cube -- lives in the file-scope device array below,
// sized for at most kNaMaxChunks chunks of kNaChunk particles.
//
// The array exists once on every GPU that loads the library and stays
// allocated until the process exits.  All calls on a device share that
// device's copy, which keeps the last call's contents; each call writes every
// byte it later reads, so nothing has to start at zero.  Two calls whose work
// overlaps on the same GPU (for example on two streams) race on the array:
// issue them on one stream, or order them with events.
//
// Keys follow the same rule as the main path: cube anchored at the per-axis
// minimum, side = largest FP32 extent (1 if below 1e-30), 21-bit FP32
// round-to-nearest quantisation, x bit most significant in each triple.
//
// The main path rejects non-finite coordinates before it builds a tree; this
// call returns before its kernels run, so it marks such input in its outputs
// instead: every key becomes BH_NOALLOC_BAD_KEY (a value no 63-bit key takes)
// and the cube becomes NaN.  Arguments that would make a kernel read or write
// out of place -- host memory, another device's memory, misaligned pointers
// -- are rejected on the host before any launch.
#include <mutex>
#include <string>

#include "bh.h"

namespace bh {
void set_last_error(const std::string &msg);  // message for bh_last_error()
}

namespace {

constexpr int kNaChunk = 4096;
constexpr int kNaThreads = 256;
constexpr int kNaMaxChunks = 4096;  // n <= 4096 * 4096 = 16,777,216
constexpr int kNaMaxDevices = 64;

struct NaBox {
    float mn[3];
    float mx[3];
    int bad;  // particles of the chunk with a non-finite coordinate
    int pad;
};

struct NaScratch {
    NaBox part[kNaMaxChunks];  // one box per chunk
    float cube[5];             // lo[3], side, scale
    int bad;                   // non-finite coordinates anywhere in the input
    int pad[2];
};

// 128 KiB + 32 bytes per GPU
static __device__ __align__(256) NaScratch g_na_scratch;

std::mutex g_na_mu;
NaScratch *g_na_addr[kNaMaxDevices] = {nullptr};

__device__ __forceinline__ float na_warp_min(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float na_warp_max(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Block min/max of 6 values, result in thread 0.
__device__ void na_block_box(float mn[3], float mx[3])
{
    __shared__ float smn[3][32], smx[3][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int a = 0; a < 3; ++a) {
        mn[a] = na_warp_min(mn[a]);
        mx[a] = na_warp_max(mx[a]);
        if (lane == 0) {
            smn[a][w] = mn[a];
            smx[a][w] = mx[a];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < nw; ++k)
            for (int a = 0; a < 3; ++a) {
                mn[a] = fminf(mn[a], smn[a][k]);
                mx[a] = fmaxf(mx[a], smx[a][k]);
            }
    }
}

__global__ void __launch_bounds__(kNaThreads)
k_na_box(const float4 *__restrict__ pos, int n, NaScratch *__restrict__ s)
{
    const int base = blockIdx.x * kNaChunk;
    const int cnt = min(kNaChunk, n - base);
    float mn[3], mx[3];
    for (int a = 0; a < 3; ++a) {
        mn[a] = __int_as_float(0x7f800000);
        mx[a] = __int_as_float(0xff800000);
    }
    int bad = 0;
    for (int i = threadIdx.x; i < cnt; i += kNaThreads) {
        const float4 p = pos[base + i];
        bad += !(isfinite(p.x) && isfinite(p.y) && isfinite(p.z));
        mn[0] = fminf(mn[0], p.x); mx[0] = fmaxf(mx[0], p.x);
        mn[1] = fminf(mn[1], p.y); mx[1] = fmaxf(mx[1], p.y);
        mn[2] = fminf(mn[2], p.z); mx[2] = fmaxf(mx[2], p.z);
    }
    bad = __syncthreads_count(bad != 0);
    na_block_box(mn, mx);
    if (threadIdx.x == 0) {
        NaBox b;
        for (int a = 0; a < 3; ++a) { b.mn[a] = mn[a]; b.mx[a] = mx[a]; }
        b.bad = bad;
        b.pad = 0;
        s->part[blockIdx.x] = b;
    }
}

__global__ void __launch_bounds__(kNaThreads)
k_na_cube(int nchunks, NaScratch *__restrict__ s, float *__restrict__ cube_out)
{
    float mn[3], mx[3];
    for (int a = 0; a < 3; ++a) {
        mn[a] = __int_as_float(0x7f800000);
        mx[a] = __int_as_float(0xff800000);
    }
    int bad = 0;
    for (int k = threadIdx.x; k < nchunks; k += kNaThreads) {
        const NaBox b = s->part[k];
        bad += b.bad;
        for (int a = 0; a < 3; ++a) {
            mn[a] = fminf(mn[a], b.mn[a]);
            mx[a] = fmaxf(mx[a], b.mx[a]);
        }
    }
    bad = __syncthreads_count(bad != 0);
    na_block_box(mn, mx);
    if (threadIdx.x == 0 && bad) {
        // no cube exists for non-finite input: mark it (keys likewise)
        s->bad = 1;
        if (cube_out)
            for (int a = 0; a < 4; ++a) cube_out[a] = __int_as_float(0x7fc00000);
    } else if (threadIdx.x == 0) {
        s->bad = 0;
        float side = 0.f;
        for (int a = 0; a < 3; ++a) {
            const float e = __fsub_rn(mx[a], mn[a]);
            if (e > side) side = e;
        }
        if (!(side >= 1e-30f)) side = 1.0f;
        const float scale = __fdiv_rn(2097152.0f, side);
        for (int a = 0; a < 3; ++a) s->cube[a] = mn[a];
        s->cube[3] = side;
        s->cube[4] = scale;
        if (cube_out) {
            for (int a = 0; a < 3; ++a) cube_out[a] = mn[a];
            cube_out[3] = side;
        }
    }
}

__device__ __forceinline__ uint32_t na_quantise(float x, float lo, float scale)
{
    const float f = floorf(__fmul_rn(__fsub_rn(x, lo), scale));
    if (!(f > 0.0f)) return 0u;
    if (f >= 2097151.0f) return 2097151u;
    return (uint32_t)f;
}

__device__ __forceinline__ uint64_t na_spread3(uint32_t v)
{
    uint64_t x = v & 0x1fffffu;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

__global__ void __launch_bounds__(kNaThreads)
k_na_keys(const float4 *__restrict__ pos, int n, const NaScratch *__restrict__ s,
          uint64_t *__restrict__ keys)
{
    const float lx = s->cube[0], ly = s->cube[1], lz = s->cube[2], scale = s->cube[4];
    const bool bad = s->bad != 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (bad) {
            keys[i] = BH_NOALLOC_BAD_KEY;
            continue;
        }
        const float4 p = pos[i];
        keys[i] = (na_spread3(na_quantise(p.x, lx, scale)) << 2) |
                  (na_spread3(na_quantise(p.y, ly, scale)) << 1) | na_spread3(na_quantise(p.z, lz, scale));
    }
}

int na_fail(int code, const std::string &m)
{
    bh::set_last_error(m);
    return code;
}

// BH_OK if p is memory that kernels on device `dev` can read and write in
// place (device memory of that device, or managed memory) and is aligned to
// `align` bytes; otherwise a message in bh_last_error and BH_ERR_INVALID.
// cudaPointerGetAttributes allocates nothing.
int na_check_ptr(const void *p, const char *what, int dev, uintptr_t align)
{
    if ((uintptr_t)p % align != 0)
        return na_fail(BH_ERR_INVALID, std::string(what) + " must be aligned to " +
                                           std::to_string((unsigned long long)align) + " bytes");
    cudaPointerAttributes at;
    const cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return na_fail(BH_ERR_INVALID, std::string(what) + ": not a pointer the CUDA runtime knows (" +
                                           cudaGetErrorString(e) + ")");
    }
    if (at.type == cudaMemoryTypeManaged) return BH_OK;
    if (at.type == cudaMemoryTypeDevice && at.device == dev) return BH_OK;
    return na_fail(BH_ERR_INVALID, std::string(what) +
                                       " must be device memory of the current device (or managed memory)");
}

}  // namespace

extern "C" {

int bh_morton_keys_noalloc(const float *pos_mass, int64_t n, uint64_t *keys, float *cube,
                           void *stream)
{
    if (!pos_mass || !keys) return na_fail(BH_ERR_INVALID, "null pos_mass or keys");
    if (n < 1 || n > (int64_t)kNaChunk * kNaMaxChunks)
        return na_fail(BH_ERR_INVALID, "n must be in [1, " + std::to_string((int64_t)kNaChunk * kNaMaxChunks) +
                                           "] (the static scratch holds " + std::to_string(kNaMaxChunks) +
                                           " chunks of " + std::to_string(kNaChunk) + ")");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(BH_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kNaMaxDevices) return na_fail(BH_ERR_INVALID, "device ordinal out of range");
    NaScratch *s = nullptr;
    {
        // set-up, once per device, with that device current: the array's
        // name is a host-side stand-in, the kernels need its device address
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_na_scratch);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return na_fail(BH_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            }
            g_na_addr[dev] = static_cast<NaScratch *>(p);
        }
        s = g_na_addr[dev];
    }
    // pos_mass is read as float4, keys written as 64-bit words, cube as floats
    int rc = na_check_ptr(pos_mass, "pos_mass", dev, 16);
    if (rc == BH_OK) rc = na_check_ptr(keys, "keys", dev, 8);
    if (rc == BH_OK && cube) rc = na_check_ptr(cube, "cube", dev, 4);
    if (rc != BH_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int ni = (int)n;
    const int nchunks = (ni + kNaChunk - 1) / kNaChunk;
    const float4 *pos = reinterpret_cast<const float4 *>(pos_mass);
    k_na_box<<<nchunks, kNaThreads, 0, st>>>(pos, ni, s);
    k_na_cube<<<1, kNaThreads, 0, st>>>(nchunks, s, cube);
    k_na_keys<<<(ni + kNaThreads - 1) / kNaThreads < 65535 ? (ni + kNaThreads - 1) / kNaThreads : 65535,
                kNaThreads, 0, st>>>(pos, ni, s, keys);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(BH_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return BH_OK;
}

}  // extern "C"
