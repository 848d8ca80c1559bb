// build_kernels.cu -- per-step O(n) kernels of the Barnes-Hut hot path:
// leapfrog kick/drift fused with the bounding-box / root reductions, Morton
// keys, the gather into Morton order, the octree topology, the bottom-up
// centre-of-mass pass, the closing kick, diagnostics and the tree export.
//
// Paper: Dekate et al., arXiv:1109.5190.  Section I: the particles are grouped
// in nested cubes, each split into eight until every leaf holds a single
// particle, with a centre of mass per cube; Section III: the tree is rebuilt
// from all positions in every iteration (a global barrier), then forces are
// computed.
// Every kernel here is HBM-bound streaming work (no tensor cores): loads are
// coalesced float4, one block per chunk of <= 4096 particles of one system.
#include "bh.h"
#include "bh_internal.cuh"

namespace bh {

thread_local int g_launches = 0;

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ bool halted(const Small *sm) { return sm->status != ST_OK; }

// Deterministic block reduction helpers (fixed shuffle tree, then warps in
// order by thread 0): results depend only on blockDim and the inputs.
template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
    return v;
}
__device__ __forceinline__ float warp_min(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_down_sync(FULL, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(FULL, v, o));
    return v;
}

struct BoxAcc {
    float mn[3], mx[3];
    double m, s[3];
};

__device__ __forceinline__ void box_init(BoxAcc &b)
{
    for (int a = 0; a < 3; ++a) {
        b.mn[a] = __int_as_float(0x7f800000);   // +inf
        b.mx[a] = __int_as_float(0xff800000);   // -inf
        b.s[a] = 0.0;
    }
    b.m = 0.0;
}

// Reduces BoxAcc over the block; the result is valid in thread 0.
__device__ BoxAcc box_block_reduce(BoxAcc b)
{
    __shared__ float smn[3][32], smx[3][32];
    __shared__ double sm[4][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int a = 0; a < 3; ++a) {
        b.mn[a] = warp_min(b.mn[a]);
        b.mx[a] = warp_max(b.mx[a]);
        b.s[a] = warp_sum(b.s[a]);
    }
    b.m = warp_sum(b.m);
    if (lane == 0) {
        for (int a = 0; a < 3; ++a) {
            smn[a][w] = b.mn[a];
            smx[a][w] = b.mx[a];
            sm[a][w] = b.s[a];
        }
        sm[3][w] = b.m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < nw; ++k) {
            for (int a = 0; a < 3; ++a) {
                b.mn[a] = fminf(b.mn[a], smn[a][k]);
                b.mx[a] = fmaxf(b.mx[a], smx[a][k]);
                b.s[a] += sm[a][k];
            }
            b.m += sm[3][k];
        }
    }
    return b;
}

// ------------------------------------------------ kick + drift + box (A8/A1)

// Leapfrog opening half: v += a dt/2, x += v dt (after saving x, v for a
// possible roll-back), fused with the per-chunk partial reductions of the new
// positions: FP32 min/max (exact) and FP64 mass and mass-weighted position
// sums (root centre of mass).
__global__ void __launch_bounds__(kChunkThreads)
k_kick_drift_box(const int4 *__restrict__ chunks, const SysStatic *__restrict__ sys,
                 const int *__restrict__ mode, ChunkPart *__restrict__ parts,
                 const Small *__restrict__ sm)
{
    if (halted(sm)) return;
    const int4 c = chunks[blockIdx.x];
    const SysStatic S = sys[c.x];
    const bool kdk = mode[c.x] == MODE_KDK;
    const int loc0 = c.y - S.start;
    BoxAcc b;
    box_init(b);
    for (int k = 0; k < kItems; ++k) {
        const int i = k * kChunkThreads + threadIdx.x;
        if (i >= c.z) break;
        const int li = loc0 + i;
        float4 p = S.pos[li];
        if (kdk) {
            float4 v = S.vel[li];
            const float4 a = S.acc[li];
            S.bpos[li] = p;
            S.bvel[li] = v;
            v.x = fmaf(a.x, S.half_dt, v.x);
            v.y = fmaf(a.y, S.half_dt, v.y);
            v.z = fmaf(a.z, S.half_dt, v.z);
            p.x = fmaf(v.x, S.dt, p.x);
            p.y = fmaf(v.y, S.dt, p.y);
            p.z = fmaf(v.z, S.dt, p.z);
            S.vel[li] = v;
            S.pos[li] = p;
        }
        b.mn[0] = fminf(b.mn[0], p.x); b.mx[0] = fmaxf(b.mx[0], p.x);
        b.mn[1] = fminf(b.mn[1], p.y); b.mx[1] = fmaxf(b.mx[1], p.y);
        b.mn[2] = fminf(b.mn[2], p.z); b.mx[2] = fmaxf(b.mx[2], p.z);
        const double m = (double)p.w;
        b.m += m;
        b.s[0] = fma(m, (double)p.x, b.s[0]);
        b.s[1] = fma(m, (double)p.y, b.s[1]);
        b.s[2] = fma(m, (double)p.z, b.s[2]);
    }
    b = box_block_reduce(b);
    if (threadIdx.x == 0) {
        ChunkPart out;
        for (int a = 0; a < 3; ++a) { out.mn[a] = b.mn[a]; out.mx[a] = b.mx[a]; }
        out.pad[0] = out.pad[1] = 0.f;
        out.m = b.m; out.sx = b.s[0]; out.sy = b.s[1]; out.sz = b.s[2];
        parts[blockIdx.x] = out;
    }
}

// Per system: combine the chunk partials in a fixed order; derive the key
// cube (lo = per-axis minimum, side = largest FP32 extent, 1 if < 1e-30,
// scale = RN32(2^21 / side)) and the FP64 root mass and centre of mass.
__global__ void __launch_bounds__(256)
k_box_final(const SysStatic *__restrict__ sys, SysDyn *__restrict__ dyn,
            const ChunkPart *__restrict__ parts, const Small *__restrict__ sm)
{
    if (halted(sm)) return;
    const SysStatic S = sys[blockIdx.x];
    BoxAcc b;
    box_init(b);
    for (int k = threadIdx.x; k < S.nchunk; k += blockDim.x) {
        const ChunkPart p = parts[S.chunk0 + k];
        for (int a = 0; a < 3; ++a) {
            b.mn[a] = fminf(b.mn[a], p.mn[a]);
            b.mx[a] = fmaxf(b.mx[a], p.mx[a]);
        }
        b.m += p.m; b.s[0] += p.sx; b.s[1] += p.sy; b.s[2] += p.sz;
    }
    b = box_block_reduce(b);
    if (threadIdx.x == 0) {
        SysDyn d;
        float side = 0.0f;
        for (int a = 0; a < 3; ++a) {
            const float e = __fsub_rn(b.mx[a], b.mn[a]);
            if (e > side) side = e;
            d.lo[a] = b.mn[a];
        }
        if (!(side >= 1e-30f)) side = 1.0f;
        d.side = side;
        d.scale = __fdiv_rn(2097152.0f, side);
        d.mtot = b.m;
        for (int a = 0; a < 3; ++a) d.mx[a] = b.s[a];
        d.root_m = (float)b.m;
        for (int a = 0; a < 3; ++a) d.root_com[a] = (float)(b.s[a] / b.m);
        d.pad = 0.f;
        dyn[blockIdx.x] = d;
    }
}

// ----------------------------------------------------------- keys (A2)

__device__ __forceinline__ uint32_t quantise(float x, float lo, float scale)
{
    const float d = __fsub_rn(x, lo);
    const float t = __fmul_rn(d, scale);
    const float f = floorf(t);
    if (!(f > 0.0f)) return 0u;
    if (f >= 2097151.0f) return 2097151u;
    return (uint32_t)f;
}

// Spreads the 21 low bits of v so bit b lands at bit 3b.
__device__ __forceinline__ uint64_t spread3(uint32_t v)
{
    uint64_t x = v & 0x1fffffu;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

// Key of every particle in input order, value = its virtual id, so the stable
// radix sort orders equal keys by input index.
__global__ void __launch_bounds__(kWideThreads)
k_keys(const int4 *__restrict__ chunks, const SysStatic *__restrict__ sys,
       const SysDyn *__restrict__ dyn, uint64_t *__restrict__ key, uint32_t *__restrict__ val,
       const Small *__restrict__ sm)
{
    if (halted(sm)) return;
    const int4 c = chunks[blockIdx.x];
    const SysStatic S = sys[c.x];
    const SysDyn D = dyn[c.x];
    const int loc0 = c.y - S.start;
    for (int k = 0; k < kWideItems; ++k) {
        const int i = k * kWideThreads + threadIdx.x;
        if (i >= c.z) break;
        const float4 p = S.pos[loc0 + i];
        const uint32_t qx = quantise(p.x, D.lo[0], D.scale);
        const uint32_t qy = quantise(p.y, D.lo[1], D.scale);
        const uint32_t qz = quantise(p.z, D.lo[2], D.scale);
        key[c.y + i] = (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
        val[c.y + i] = (uint32_t)(c.y + i);
    }
}

// ----------------------------------------------------------- permute (A4)

__global__ void __launch_bounds__(kWideThreads)
k_permute(const int4 *__restrict__ chunks, const SysStatic *__restrict__ sys,
          const uint32_t *__restrict__ sid, float4 *__restrict__ spos,
          const Small *__restrict__ sm)
{
    if (halted(sm)) return;
    const int4 c = chunks[blockIdx.x];
    const SysStatic S = sys[c.x];
    for (int k = 0; k < kWideItems; ++k) {
        const int i = k * kWideThreads + threadIdx.x;
        if (i >= c.z) break;
        const int j = c.y + i;
        spos[j] = __ldg(&S.pos[(int)sid[j] - S.start]);
    }
}

// ---------------------------------------------------------- topology (A5)

// Number of leading octal digits (levels) two keys share: 0..21.
__device__ __forceinline__ int common_levels(uint64_t a, uint64_t b)
{
    const uint64_t x = a ^ b;
    if (!x) return kLevels;
    const int p = 63 - __clzll((long long)x);
    return (kLevels - 1) - p / 3;
}

// For sorted particle j of a system [a, b): dprev / dnext = levels shared
// with its neighbours (-1 at the system's ends).  The cells that start at j
// are the levels dprev+1 .. 21; such a cell is a node iff its parent holds
// >= 2 particles, i.e. iff level - 1 <= max(dprev, dnext); the deepest of
// them is a leaf (one particle, or the level-21 bucket of equal keys).
struct Span {
    int dprev, dnext, lmax, cnt;
    int lo, hi;  // levels of the nodes the bottom-up pass computes (lo > hi: none)
};

// Sorted keys read straight from global memory.
struct GlobalKeys {
    const uint64_t *__restrict__ g;
    __device__ __forceinline__ uint64_t operator[](int p) const { return g[p]; }
};

// Sorted keys with the run key[s0 .. s1) staged in shared memory (a block's
// chunk and its two neighbours): the searches of the many small cells stay on
// chip, and only cells reaching past the chunk read global memory.
struct StagedKeys {
    const uint64_t *__restrict__ g;
    const uint64_t *s;
    int s0, s1;
    __device__ __forceinline__ uint64_t operator[](int p) const
    {
        return (p >= s0 && p < s1) ? s[p - s0] : g[p];
    }
};

template <class Keys>
__device__ __forceinline__ Span node_span(const Keys &key, int j, int a, int b)
{
    Span s;
    const uint64_t kj = key[j];
    s.dprev = (j == a) ? -1 : common_levels(key[j - 1], kj);
    s.dnext = (j == b - 1) ? -1 : common_levels(kj, key[j + 1]);
    if (s.dprev >= kLevels) {
        s.lmax = s.dprev;
        s.cnt = 0;
        s.lo = 1;
        s.hi = 0;
    } else {
        s.lmax = min(kLevels, max(s.dprev, s.dnext) + 1);
        s.cnt = s.lmax - s.dprev;
        // the root is written by the topology pass, and so is the deepest node
        // when it is a one-particle leaf (it is a bucket only if dnext = 21)
        s.lo = max(s.dprev + 1, 1);
        s.hi = s.lmax > s.dnext ? s.lmax - 1 : s.lmax;
    }
    return s;
}

__global__ void __launch_bounds__(kWideThreads)
k_topo_count(const int4 *__restrict__ chunks, const SysStatic *__restrict__ sys,
             const uint64_t *__restrict__ key, uint32_t *__restrict__ ncount,
             Small *__restrict__ sm)
{
    if (halted(sm)) return;
    __shared__ unsigned h[kNumLevels];
    if (threadIdx.x < kNumLevels) h[threadIdx.x] = 0;
    __syncthreads();
    const int4 c = chunks[blockIdx.x];
    const SysStatic S = sys[c.x];
    for (int k = 0; k < kWideItems; ++k) {
        const int i = k * kWideThreads + threadIdx.x;
        if (i >= c.z) break;
        const int j = c.y + i;
        const Span s = node_span(GlobalKeys{key}, j, S.start, S.start + S.n);
        ncount[j] = (uint32_t)s.cnt;
        for (int l = s.lo; l <= s.hi; ++l) atomicAdd(&h[l], 1u);
    }
    __syncthreads();
    if (threadIdx.x < kNumLevels && h[threadIdx.x])
        atomicAdd(&sm->level_cnt[threadIdx.x], h[threadIdx.x]);
}

// Node count check and per-level list offsets (one thread).
__global__ void k_level_offsets(Small *__restrict__ sm, const uint32_t *__restrict__ noff,
                                int n_total, unsigned cap)
{
    if (halted(sm) || threadIdx.x != 0) return;
    const unsigned M = noff[n_total];
    sm->M = M;
    if (M > cap) {
        sm->needed = M;
        sm->status = ST_CAPACITY;
        return;
    }
    unsigned off = 0;
    for (int l = 0; l < kNumLevels; ++l) {
        sm->level_off[l] = off;
        off += sm->level_cnt[l];
    }
    sm->level_off[kNumLevels] = off;
}

// First index e in [lo, b] whose key leaves the level-l cell of kj (all
// indices below lo are known to be inside): galloping then bisection.
template <class Keys>
__device__ __forceinline__ int cell_end(const Keys &key, uint64_t kj, int lo, int b, int l)
{
    const int sh = 3 * (kLevels - l);
    int step = 1, hi;
    for (;;) {
        const int p = lo + step - 1;
        if (p >= b) { hi = b; break; }
        if (((key[p] ^ kj) >> sh) != 0) { hi = p; break; }
        lo = p + 1;
        step <<= 1;
    }
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (((key[mid] ^ kj) >> sh) != 0) hi = mid; else lo = mid + 1;
    }
    return lo;
}

__device__ __forceinline__ float pow2_neg(int l) { return __int_as_float((127 - l) << 23); }

// b_max rule (BH_OPEN_BMAX): b_max^2 of a cell, the squared distance from its
// centre of mass to the farthest corner of its cube.  Per axis the cube is
// [c, c + s], c = lo + q s, s = side 2^-l, q the cell's integer position at
// level l (the key prefix de-interleaved: bit 2 of each octal digit is x,
// bit 1 y, bit 0 z); the farther face is max(com - c, (c + s) - com).  FP64,
// every operation rounded on its own.
__device__ __noinline__ double cell_bmax2(uint64_t key, int l, const SysDyn &D, double cx,
                                          double cy, double cz)
{
    const uint64_t pre = key >> (3 * (kLevels - l));
    unsigned q[3] = {0u, 0u, 0u};
    for (int b = 0; b < l; ++b) {
        const unsigned digit = (unsigned)(pre >> (3 * b)) & 7u;
        q[0] |= ((digit >> 2) & 1u) << b;
        q[1] |= ((digit >> 1) & 1u) << b;
        q[2] |= (digit & 1u) << b;
    }
    const double s = __dmul_rn((double)D.side, __longlong_as_double((long long)(1023 - l) << 52));
    const double com[3] = {cx, cy, cz};
    double e2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double c = __dadd_rn((double)D.lo[a], __dmul_rn((double)q[a], s));
        const double lo_gap = __dsub_rn(com[a], c);
        const double hi_gap = __dsub_rn(__dadd_rn(c, s), com[a]);
        const double e = lo_gap > hi_gap ? lo_gap : hi_gap;
        e2 = __dadd_rn(e2, __dmul_rn(e, e));
    }
    return e2;
}

// The walk's FP32 threshold for b_max^2: accept iff d^2 > b_max^2 / theta^2,
// rounded once; kept finite so that it never reads as the bucket marker.
__device__ __forceinline__ float bmax_crit(double bm2, double theta2)
{
    return fminf(__double2float_rn(__ddiv_rn(bm2, theta2)), 3.40282347e38f);
}

// Writes every node that starts at a particle: skip pointer (the first node
// starting at the cell's end particle), first, count, level and opening
// threshold, plus its slot in its level's list.  The root's centre of mass
// comes from the FP64 reduction (or the particle itself for a one-particle
// system); every other centre of mass is written by the bottom-up pass.
// Each 4096-particle chunk is split over kTopoSplit blocks of kTopoThreads, so
// the grid spreads evenly over the SMs (one 1024-thread block per chunk left
// the second of two waves two-thirds full).
constexpr int kTopoSplit = 4;
constexpr int kTopoThreads = 256;
constexpr int kTopoSpan = kChunk / kTopoSplit;        // 1024 particles per block
constexpr int kTopoItems = kTopoSpan / kTopoThreads;  // 4 per thread

__global__ void __launch_bounds__(kTopoThreads)
k_topo_write(const int4 *__restrict__ chunks, const SysStatic *__restrict__ sys,
             const SysDyn *__restrict__ dyn, const uint64_t *__restrict__ key,
             const uint32_t *__restrict__ noff, const float4 *__restrict__ spos,
             WNode *__restrict__ nodeW, int4 *__restrict__ nodeR, double4_32a *__restrict__ nodeD,
             uint32_t *__restrict__ nlist, double *__restrict__ nodeI, float4 *__restrict__ nodeQ,
             double *__restrict__ nodeB, Small *__restrict__ sm)
{
    if (halted(sm)) return;
    const int4 cc = chunks[blockIdx.x / kTopoSplit];
    const int part = (int)blockIdx.x % kTopoSplit;
    // this block's particles [c.y, c.y + c.z) of chunk cc
    const int4 c = make_int4(cc.x, cc.y + part * kTopoSpan, min(kTopoSpan, cc.z - part * kTopoSpan), 0);
    if (c.z <= 0) return;  // a short chunk: the whole block leaves together
    __shared__ unsigned h[kNumLevels], base[kNumLevels];
    __shared__ uint64_t skey[kTopoSpan + 2];
    if (threadIdx.x < kNumLevels) h[threadIdx.x] = 0;
    const SysStatic S = sys[c.x];
    const int a = S.start, b = S.start + S.n;
    // the block's keys and one neighbour on each side (within the system)
    const int s0 = max(c.y - 1, a), s1 = min(c.y + c.z + 1, b);
    for (int p = s0 + (int)threadIdx.x; p < s1; p += kTopoThreads) skey[p - s0] = key[p];
    __syncthreads();
    const StagedKeys K{key, skey, s0, s1};
    for (int k = 0; k < kTopoItems; ++k) {
        const int i = k * kTopoThreads + threadIdx.x;
        if (i >= c.z) break;
        const Span s = node_span(K, c.y + i, a, b);
        for (int l = s.lo; l <= s.hi; ++l) atomicAdd(&h[l], 1u);
    }
    __syncthreads();
    if (threadIdx.x < kNumLevels) {
        const unsigned cnt = h[threadIdx.x];
        base[threadIdx.x] = (cnt ? atomicAdd(&sm->level_cur[threadIdx.x], cnt) : 0u) +
                            sm->level_off[threadIdx.x];
        h[threadIdx.x] = 0;
    }
    __syncthreads();
    const SysDyn D = dyn[c.x];
    for (int k = 0; k < kTopoItems; ++k) {
        const int i = k * kTopoThreads + threadIdx.x;
        if (i >= c.z) break;
        const int j = c.y + i;
        const Span s = node_span(K, j, a, b);
        if (s.cnt == 0) continue;
        const uint64_t kj = K[j];
        const unsigned nb = noff[j];
        int end = j + 1;
        for (int l = s.lmax; l > s.dprev; --l) {
            const unsigned n = nb + (unsigned)(l - s.dprev - 1);
            if (l <= s.dnext) end = cell_end(K, kj, max(end, j + 2), b, l);
            else end = j + 1;
            const int count = end - j;
            float crit;
            if (count == 1) {
                crit = kLeafCrit;
            } else if (l == kLevels) {
                crit = kBucketCrit;
            } else {
                const float sl = __fmul_rn(D.side, pow2_neg(l));
                crit = __fmul_rn(__fmul_rn(sl, sl), S.inv_theta2);
            }
            nodeR[n] = make_int4(j, count, l, c.x);
            // the walk's loop bound: every skip pointer lies past its node and
            // within the system's nodes (true by construction; checked here so
            // that the walk itself need not)
            const unsigned skip = noff[end];
            if (skip <= n || skip > noff[b]) atomicExch(&sm->status, ST_WALK_LIMIT);
            // low part 0 with scale 2^0 until the centre-of-mass pass fills it
            nodeW[n].b = make_uint4(__float_as_uint(crit), skip, 0u, 127u << 23);
            if (l >= s.lo && l <= s.hi) {
                nlist[base[l] + atomicAdd(&h[l], 1u)] = n;
            } else if (l > 0) {  // one-particle leaf: the particle itself
                const float4 p = spos[j];
                nodeW[n].a = p;
                nodeD[n] = make_double4_32a(p.w, p.x, p.y, p.z);
                if (nodeI) {  // no second moments about itself
                    for (int q = 0; q < 6; ++q) nodeI[6 * (size_t)n + q] = 0.0;
                    nodeQ[2 * (size_t)n] = make_float4(0.f, 0.f, 0.f, 0.f);
                    nodeQ[2 * (size_t)n + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            if (l == 0) {
                if (count == 1) {
                    const float4 p = spos[j];
                    nodeW[n].a = p;
                    nodeD[n] = make_double4_32a(p.w, p.x, p.y, p.z);
                    if (nodeI) {
                        for (int q = 0; q < 6; ++q) nodeI[6 * (size_t)n + q] = 0.0;
                        nodeQ[2 * (size_t)n] = make_float4(0.f, 0.f, 0.f, 0.f);
                        nodeQ[2 * (size_t)n + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                } else {
                    const double cx = D.mx[0] / D.mtot, cy = D.mx[1] / D.mtot, cz = D.mx[2] / D.mtot;
                    const float hx = (float)cx, hy = (float)cy, hz = (float)cz;
                    nodeW[n].a = make_float4(hx, hy, hz, (float)D.mtot);
                    if (nodeB && crit != kBucketCrit) {
                        const double bm2 = cell_bmax2(kj, 0, D, cx, cy, cz);
                        nodeB[n] = bm2;
                        crit = bmax_crit(bm2, S.theta2);
                    }
                    nodeW[n].b = wn_pack(crit, (int)skip, cx, cy, cz, hx, hy, hz);
                    nodeD[n] = make_double4_32a(D.mtot, cx, cy, cz);
                }
            }
        }
    }
}

// ------------------------------------------------- centre of mass (A6)

// Bottom-up, level by level (deepest first), in FP64, over the nodes of each
// level that are not one-particle leaves (those, and the roots, are written by
// the topology pass): a bucket sums its particles; an internal node sums its
// children (first child = next node, then skip pointers):
// M = sum m_c, com = sum m_c com_c / M.  The FP64 result is kept (nodeD) and
// split into an FP32 high part and a packed low part for the walk.
// Quadrupole mode: second moments I_ab = sum m r_a r_b about the node's centre
// of mass (cx, cy, cz), in FP64: a bucket sums its particles; an internal node
// sums its children's moments moved to its own centre (parallel axes:
// I_child + m_child (c_child - c)(c_child - c)^T), in a second pass over the
// children once the centre is known.  Also writes the FP32 copy for the walk.
__device__ __noinline__ void second_moments(unsigned n, int4 C, float crit, int skip, double cx,
                                            double cy, double cz,
                                            const float4 *__restrict__ spos,
                                            const WNode *__restrict__ nodeW,
                                            const double4_32a *__restrict__ nodeD,
                                            double *__restrict__ nodeI, float4 *__restrict__ nodeQ)
{
    double I[6] = {0, 0, 0, 0, 0, 0};
    if (crit == kBucketCrit) {
        for (int q = C.x; q < C.x + C.y; ++q) {
            const float4 p = spos[q];
            const double m = p.w, r0 = p.x - cx, r1 = p.y - cy, r2 = p.z - cz;
            I[0] += m * r0 * r0; I[1] += m * r1 * r1; I[2] += m * r2 * r2;
            I[3] += m * r0 * r1; I[4] += m * r0 * r2; I[5] += m * r1 * r2;
        }
    } else {
        for (int ch = (int)n + 1; ch < skip; ch = wn_skip(nodeW[ch].b)) {
            const double4_32a d = nodeD[ch];
            const double *Ic = nodeI + 6 * (size_t)ch;
            const double r0 = d.y - cx, r1 = d.z - cy, r2 = d.w - cz;
            I[0] += Ic[0] + d.x * r0 * r0; I[1] += Ic[1] + d.x * r1 * r1;
            I[2] += Ic[2] + d.x * r2 * r2; I[3] += Ic[3] + d.x * r0 * r1;
            I[4] += Ic[4] + d.x * r0 * r2; I[5] += Ic[5] + d.x * r1 * r2;
        }
    }
    for (int q = 0; q < 6; ++q) nodeI[6 * (size_t)n + q] = I[q];
    nodeQ[2 * (size_t)n] = make_float4((float)I[0], (float)I[1], (float)I[2], (float)I[3]);
    nodeQ[2 * (size_t)n + 1] = make_float4((float)I[4], (float)I[5], 0.f, 0.f);
}

// b_max rule only (else nodeB is null): what the centre-of-mass pass needs to
// rewrite a cell's threshold once its centre is known
struct ComRule {
    const SysStatic *sys;
    const SysDyn *dyn;
    const uint64_t *key;  // sorted keys
    double *nodeB;        // FP64 b_max^2 per cell, read by the walk's tie test
};

// EXTRA: the b_max rule or quadrupole moments are on (their arrays non-null);
// without them the kernels compile without those paths, in fewer registers.
template <bool EXTRA>
__device__ __forceinline__ void com_node(unsigned n, const float4 *__restrict__ spos,
                                         WNode *__restrict__ nodeW, const int4 *__restrict__ nodeR,
                                         double4_32a *__restrict__ nodeD, double *__restrict__ nodeI,
                                         float4 *__restrict__ nodeQ, const ComRule &R)
{
    const int4 C = nodeR[n];  // first, count, level
    const uint4 B = nodeW[n].b;
    const float crit = wn_crit(B);
    const int skip = wn_skip(B);
    double M = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
    if (crit == kBucketCrit) {
        for (int q = C.x; q < C.x + C.y; ++q) {
            const float4 p = spos[q];
            const double m = p.w;
            M += m;
            sx += m * (double)p.x;
            sy += m * (double)p.y;
            sz += m * (double)p.z;
        }
    } else {
        for (int ch = (int)n + 1; ch < skip; ch = wn_skip(nodeW[ch].b)) {
            const double4_32a d = nodeD[ch];
            M += d.x;
            sx += d.x * d.y;
            sy += d.x * d.z;
            sz += d.x * d.w;
        }
    }
    const double inv = 1.0 / M;
    const double cx = sx * inv, cy = sy * inv, cz = sz * inv;
    const float hx = (float)cx, hy = (float)cy, hz = (float)cz;
    nodeD[n] = make_double4_32a(M, cx, cy, cz);
    nodeW[n].a = make_float4(hx, hy, hz, (float)M);
    float crit_w = crit;
    if (EXTRA && R.nodeB && crit != kBucketCrit) {  // a cell (theta > 0): b_max threshold
        const double bm2 = cell_bmax2(R.key[C.x], C.z, R.dyn[C.w], cx, cy, cz);
        R.nodeB[n] = bm2;
        crit_w = bmax_crit(bm2, R.sys[C.w].theta2);
    }
    nodeW[n].b = wn_pack(crit_w, skip, cx, cy, cz, hx, hy, hz);
    if (EXTRA && nodeI) second_moments(n, C, crit, skip, cx, cy, cz, spos, nodeW, nodeD, nodeI, nodeQ);
}

// One level, all blocks (the lean variant: six blocks of 256 per SM, 48 warps
// to hide the latency of each thread's chain of child loads).
template <bool EXTRA>
__global__ void __launch_bounds__(256, EXTRA ? 1 : 6)
k_com_level(int l, const uint32_t *__restrict__ nlist, const float4 *__restrict__ spos,
            WNode *__restrict__ nodeW, const int4 *__restrict__ nodeR, double4_32a *__restrict__ nodeD,
            double *__restrict__ nodeI, float4 *__restrict__ nodeQ, ComRule R,
            const Small *__restrict__ sm)
{
    if (halted(sm)) return;
    const unsigned cnt = sm->level_cnt[l];
    const unsigned off = sm->level_off[l];
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x)
        com_node<EXTRA>(nlist[off + k], spos, nodeW, nodeR, nodeD, nodeI, nodeQ, R);
}

// The deep levels l_hi .. l_lo, which hold few nodes, in one block: a block
// barrier separates the levels, so one launch replaces many near-empty ones.
template <bool EXTRA>
__global__ void __launch_bounds__(1024)
k_com_deep(int l_hi, int l_lo, const uint32_t *__restrict__ nlist, const float4 *__restrict__ spos,
           WNode *__restrict__ nodeW, const int4 *__restrict__ nodeR, double4_32a *__restrict__ nodeD,
           double *__restrict__ nodeI, float4 *__restrict__ nodeQ, ComRule R,
           const Small *__restrict__ sm)
{
    if (halted(sm)) return;
    for (int l = l_hi; l >= l_lo; --l) {
        const unsigned cnt = sm->level_cnt[l];
        const unsigned off = sm->level_off[l];
        for (unsigned k = threadIdx.x; k < cnt; k += blockDim.x)
            com_node<EXTRA>(nlist[off + k], spos, nodeW, nodeR, nodeD, nodeI, nodeQ, R);
        __syncthreads();
    }
}

// Quadrupole mode: each system's root (written by the topology pass, centre
// of mass from the FP64 reduction) gets its second moments from its children
// once level 1 is done.  One thread per system.
__global__ void k_root_moments(const SysStatic *__restrict__ sys,
                               const uint32_t *__restrict__ noff, const float4 *__restrict__ spos,
                               const WNode *__restrict__ nodeW, const int4 *__restrict__ nodeR,
                               const double4_32a *__restrict__ nodeD, double *__restrict__ nodeI,
                               float4 *__restrict__ nodeQ, const Small *__restrict__ sm)
{
    if (halted(sm) || threadIdx.x != 0) return;
    const SysStatic S = sys[blockIdx.x];
    const unsigned n = noff[S.start];
    const int4 C = nodeR[n];
    if (C.y < 2) return;  // a one-particle root is a leaf (moments zero)
    const double4_32a D = nodeD[n];
    const uint4 B = nodeW[n].b;
    second_moments(n, C, wn_crit(B), wn_skip(B), D.y, D.z, D.w, spos, nodeW, nodeD, nodeI, nodeQ);
}

// ----------------------------------------------- sibling-order copy (walk)
//
// For the sibling-order walk: every system's root at the system's index, then
// the children of each node stored next to each other, the blocks in the
// depth-first order of their parents (position of child r of node p:
// nsys + (children of the nodes before p) + r).  Child counts and positions
// come from each cell's chain of children (first child p + 1, then skip
// pointers up to p's own skip); then the records are rewritten with
// sibling-order pointers.  Each particle's walk visits the same nodes in the
// same order as in depth-first order; only where the records sit changes.

// A node has children iff it holds two or more particles above the depth cap.
__device__ __forceinline__ bool has_children(const int4 &R) { return R.y > 1 && R.z < kLevels; }

// nch[k] = children of node k (0 for leaves and buckets), for every k below
// the node capacity (0 past the last node), for the scan that follows.
__global__ void __launch_bounds__(256)
k_sib_count(const uint32_t *__restrict__ mtot, unsigned cap, const WNode *__restrict__ nodeW,
            const int4 *__restrict__ nodeR, uint32_t *__restrict__ nch,
            const Small *__restrict__ sm)
{
    if (halted(sm)) return;
    const unsigned m = *mtot;
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < cap; k += gridDim.x * blockDim.x) {
        unsigned c = 0;
        if (k < m && has_children(nodeR[k])) {
            const unsigned end = (unsigned)wn_skip(nodeW[k].b);
            for (unsigned ch = k + 1; ch < end; ch = (unsigned)wn_skip(nodeW[ch].b)) ++c;
        }
        nch[k] = c;
    }
}

// Places every node: roots at their system's index, the children of node p at
// nsys + excl[p] + r (excl = exclusive scan of nch).  lidx: depth-first ->
// sibling order; ldfs: the inverse.
__global__ void __launch_bounds__(256)
k_sib_place(const uint32_t *__restrict__ mtot, int nsys, const WNode *__restrict__ nodeW,
            const int4 *__restrict__ nodeR, const uint32_t *__restrict__ excl,
            uint32_t *__restrict__ lidx, uint32_t *__restrict__ ldfs,
            const Small *__restrict__ sm)
{
    if (halted(sm)) return;
    const unsigned m = *mtot;
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
        const int4 R = nodeR[k];
        if (R.z == 0) {
            lidx[k] = (unsigned)R.w;
            ldfs[R.w] = k;
        }
        if (!has_children(R)) continue;
        const unsigned end = (unsigned)wn_skip(nodeW[k].b);
        unsigned pos = (unsigned)nsys + excl[k];
        for (unsigned ch = k + 1; ch < end; ch = (unsigned)wn_skip(nodeW[ch].b), ++pos) {
            lidx[ch] = pos;
            ldfs[pos] = ch;
        }
    }
}

// Rewrites node k's record at its sibling-order slot.  Checks that the map is
// a bijection (ldfs[lidx[k]] == k with lidx[k] < m for every k): then the
// sibling-order pointers copy the depth-first ones one to one, and the walk
// over them visits what the depth-first walk visits and ends where it ends.
__global__ void __launch_bounds__(256)
k_sib_write(const SysStatic *__restrict__ sys, const uint32_t *__restrict__ noff, int n_total,
            const WNode *__restrict__ nodeW, const int4 *__restrict__ nodeR,
            const double4_32a *__restrict__ nodeD, const uint32_t *__restrict__ lidx,
            const uint32_t *__restrict__ ldfs, WNode *__restrict__ nodeF,
            double4_32a *__restrict__ nodeDF, Small *__restrict__ sm)
{
    if (halted(sm)) return;
    const unsigned m = noff[n_total];
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
        const unsigned me = lidx[k];
        const int4 R = nodeR[k];  // first, count, level, system
        // a bijection, with every system's root at the system's index
        if (me >= m || ldfs[me] != k || (R.z == 0 && me != (unsigned)R.w)) {
            atomicExch(&sm->status, ST_WALK_LIMIT);
            return;
        }
        const WNode W = nodeW[k];
        const float crit = wn_crit(W.b);
        const unsigned skip = (unsigned)wn_skip(W.b);
        const SysStatic &S = sys[R.w];
        const unsigned nend = noff[S.start + S.n];
        unsigned kind, target;
        if (crit == kLeafCrit) {
            kind = kSibLeaf;
            target = (unsigned)R.x;
        } else if (crit == kBucketCrit) {
            kind = kSibBucket;
            target = k;
        } else {
            if (k + 1 >= nend) {  // a cell has children (true by construction)
                atomicExch(&sm->status, ST_WALK_LIMIT);
                return;
            }
            kind = kSibCell;
            target = lidx[k + 1];  // first child: the next node in depth-first order
        }
        const unsigned next = skip < nend ? lidx[skip] : kSibEnd;
        const unsigned meta = (W.b.w & 0xff80ffffu) | ((unsigned)R.z << 16) | (kind << 21);
        WNode F;
        F.a = W.a;
        F.b = make_uint4(target, next, W.b.z, meta);
        nodeF[me] = F;
        nodeDF[me] = nodeD[k];
    }
}

// ------------------------------------------------------ closing kick (A8)

__global__ void __launch_bounds__(kWideThreads)
k_kick(const int4 *__restrict__ chunks, const SysStatic *__restrict__ sys,
       const int *__restrict__ mode, Small *__restrict__ sm)
{
    if (halted(sm)) return;
    const int4 c = chunks[blockIdx.x];
    if (blockIdx.x == 0 && threadIdx.x == 0) sm->steps_done += 1;
    if (mode[c.x] != MODE_KDK) return;
    const SysStatic S = sys[c.x];
    const int loc0 = c.y - S.start;
    for (int k = 0; k < kWideItems; ++k) {
        const int i = k * kWideThreads + threadIdx.x;
        if (i >= c.z) break;
        const int li = loc0 + i;
        float4 v = S.vel[li];
        const float4 a = S.acc[li];
        v.x = fmaf(a.x, S.half_dt, v.x);
        v.y = fmaf(a.y, S.half_dt, v.y);
        v.z = fmaf(a.z, S.half_dt, v.z);
        S.vel[li] = v;
    }
}

// Rolls back the opening kick/drift of a step that overflowed the node buffer.
__global__ void __launch_bounds__(kWideThreads)
k_restore(const int4 *__restrict__ chunks, const SysStatic *__restrict__ sys,
          const int *__restrict__ mode)
{
    const int4 c = chunks[blockIdx.x];
    if (mode[c.x] != MODE_KDK) return;
    const SysStatic S = sys[c.x];
    const int loc0 = c.y - S.start;
    for (int k = 0; k < kWideItems; ++k) {
        const int i = k * kWideThreads + threadIdx.x;
        if (i >= c.z) break;
        S.pos[loc0 + i] = S.bpos[loc0 + i];
        S.vel[loc0 + i] = S.bvel[loc0 + i];
    }
}

// Input check for device-resident inputs: finite coordinates, mass > 0.
__global__ void __launch_bounds__(kChunkThreads)
k_validate(const int4 *__restrict__ chunks, const SysStatic *__restrict__ sys,
           Small *__restrict__ sm)
{
    const int4 c = chunks[blockIdx.x];
    const SysStatic S = sys[c.x];
    const int loc0 = c.y - S.start;
    bool bad = false;
    for (int k = 0; k < kItems; ++k) {
        const int i = k * kChunkThreads + threadIdx.x;
        if (i >= c.z) break;
        const float4 p = S.pos[loc0 + i];
        const float4 v = S.vel[loc0 + i];
        bad |= !(isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && p.w > 0.f && isfinite(p.w));
        bad |= !(isfinite(v.x) && isfinite(v.y) && isfinite(v.z));
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(&sm->status, ST_BAD_INPUT);
}

// Input check of one array pair (vel may be null): finite coordinates, mass > 0.
__global__ void __launch_bounds__(256)
k_validate_arrays(const float4 *__restrict__ pos, const float4 *__restrict__ vel, int n,
                  Small *__restrict__ sm)
{
    bool bad = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 p = pos[i];
        bad |= !(isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && p.w > 0.f && isfinite(p.w));
        if (vel) {
            const float4 v = vel[i];
            bad |= !(isfinite(v.x) && isfinite(v.y) && isfinite(v.z));
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(&sm->status, ST_BAD_INPUT);
}

// ------------------------------------------------------ diagnostics (A9)

__global__ void __launch_bounds__(kChunkThreads)
k_diag_part(const int4 *__restrict__ chunks, const SysStatic *__restrict__ sys,
            DiagPart *__restrict__ parts)
{
    const int4 c = chunks[blockIdx.x];
    const SysStatic S = sys[c.x];
    const int loc0 = c.y - S.start;
    double v[9];
    for (int q = 0; q < 9; ++q) v[q] = 0.0;
    for (int k = 0; k < kItems; ++k) {
        const int i = k * kChunkThreads + threadIdx.x;
        if (i >= c.z) break;
        const float4 p = S.pos[loc0 + i];
        const float4 u = S.vel[loc0 + i];
        const float4 a = S.acc[loc0 + i];
        const double m = p.w;
        const double ux = u.x, uy = u.y, uz = u.z;
        v[0] += 0.5 * m * (ux * ux + uy * uy + uz * uz);
        v[1] += 0.5 * m * (double)a.w;
        v[2] += m * ux; v[3] += m * uy; v[4] += m * uz;
        v[5] += m;
        v[6] += m * (double)p.x; v[7] += m * (double)p.y; v[8] += m * (double)p.z;
    }
    __shared__ double sh[9][kChunkThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int q = 0; q < 9; ++q) {
        v[q] = warp_sum(v[q]);
        if (lane == 0) sh[q][w] = v[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        DiagPart out;
        for (int q = 0; q < 9; ++q) {
            double t = sh[q][0];
            for (int k = 1; k < kChunkThreads / 32; ++k) t += sh[q][k];
            out.v[q] = t;
        }
        out.pad = 0.0;
        parts[blockIdx.x] = out;
    }
}

__global__ void k_diag_final(const SysStatic *__restrict__ sys, const DiagPart *__restrict__ parts,
                             double *__restrict__ out)
{
    if (threadIdx.x != 0) return;
    const SysStatic S = sys[blockIdx.x];
    double v[9];
    for (int q = 0; q < 9; ++q) v[q] = 0.0;
    for (int k = 0; k < S.nchunk; ++k)
        for (int q = 0; q < 9; ++q) v[q] += parts[S.chunk0 + k].v[q];
    double *o = out + 8 * blockIdx.x;
    o[0] = v[0];
    o[1] = v[1];
    o[2] = v[2]; o[3] = v[3]; o[4] = v[4];
    o[5] = v[6] / v[5]; o[6] = v[7] / v[5]; o[7] = v[8] / v[5];
}

// ----------------------------------------------------------- export

__global__ void __launch_bounds__(256)
k_export(int sysid, const SysStatic *__restrict__ sys, const uint32_t *__restrict__ noff,
         const uint64_t *__restrict__ key, const uint32_t *__restrict__ sid,
         const WNode *__restrict__ nodeW, const int4 *__restrict__ nodeR,
         bh_node *__restrict__ out_nodes,
         float4 *__restrict__ out_com, uint32_t *__restrict__ out_order)
{
    const SysStatic S = sys[sysid];
    const unsigned n0 = noff[S.start], n1 = noff[S.start + S.n];
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned n = n0 + blockIdx.x * blockDim.x + threadIdx.x; n < n1; n += stride) {
        const int4 C = nodeR[n];  // first, count, level
        const int l = C.z;
        const uint64_t pre = (l == 0) ? 0ull : (key[C.x] >> (3 * (kLevels - l)));
        unsigned cm = 0;
        const uint4 B = nodeW[n].b;
        const float crit = wn_crit(B);
        if (crit != kLeafCrit && crit != kBucketCrit) {
            for (int ch = (int)n + 1; ch < wn_skip(B); ch = wn_skip(nodeW[ch].b))
                cm |= 1u << (unsigned)((key[nodeR[ch].x] >> (3 * (kLevels - l - 1))) & 7u);
        }
        if (out_nodes) {
            bh_node o;
            o.prefix = pre;
            o.first = (uint32_t)(C.x - S.start);
            o.count = (uint32_t)C.y;
            o.level = (uint8_t)l;
            o.childmask = (uint8_t)cm;
            for (int q = 0; q < 6; ++q) o.pad[q] = 0;
            out_nodes[n - n0] = o;
        }
        if (out_com) {
            const float4 A = nodeW[n].a;
            float lx, ly, lz;
            wn_lo(B, lx, ly, lz);
            out_com[n - n0] = make_float4(A.x + lx, A.y + ly, A.z + lz, A.w);
        }
    }
    if (out_order) {
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.n; i += stride)
            out_order[i] = sid[S.start + i] - (uint32_t)S.start;
    }
}

}  // namespace

// ------------------------------------------------------------- launchers

void launch_kick_drift_bbox(const BuildBufs &b, cudaStream_t st)
{
    k_kick_drift_box<<<b.nchunks, kChunkThreads, 0, st>>>(b.chunks, b.sys, b.mode, b.parts, b.small);
    k_box_final<<<b.nsys, 256, 0, st>>>(b.sys, b.dyn, b.parts, b.small);
    g_launches += 2;
}

void launch_keys(const BuildBufs &b, cudaStream_t st)
{
    k_keys<<<b.nchunks, kWideThreads, 0, st>>>(b.chunks, b.sys, b.dyn, b.key0, b.val0, b.small);
    g_launches += 1;
}

void launch_permute(const BuildBufs &b, cudaStream_t st)
{
    k_permute<<<b.nchunks, kWideThreads, 0, st>>>(b.chunks, b.sys, b.val0, b.spos, b.small);
    g_launches += 1;
}

void launch_topology(const BuildBufs &b, cudaStream_t st)
{
    k_topo_count<<<b.nchunks, kWideThreads, 0, st>>>(b.chunks, b.sys, b.key0, b.ncount, b.small);
    g_launches += 1;
    launch_scan(b.ncount, b.noff, b.n_total, b.scan_part, b.noff + b.n_total, &b.small->status, st);
    k_level_offsets<<<1, 32, 0, st>>>(b.small, b.noff, b.n_total, b.node_cap);
    k_topo_write<<<b.nchunks * kTopoSplit, kTopoThreads, 0, st>>>(
        b.chunks, b.sys, b.dyn, b.key0, b.noff, b.spos, b.nodeW, b.nodeR, b.nodeD, b.nlist,
        b.nodeI, b.nodeQ, b.nodeB, b.small);
    g_launches += 2;
}

void launch_com(const BuildBufs &b, cudaStream_t st)
{
    const ComRule R{b.sys, b.dyn, b.key0, b.nodeB};
    const bool extra = b.nodeB || b.nodeI;
    // full occupancy: short per-thread chains of child loads
    const int grid = b.nsm * (extra ? 8 : 6);
    int l = kLevels;
    if (b.deep_cut <= kLevels) {
        auto *deep = extra ? k_com_deep<true> : k_com_deep<false>;
        deep<<<1, 1024, 0, st>>>(kLevels, b.deep_cut, b.nlist, b.spos, b.nodeW, b.nodeR, b.nodeD,
                                 b.nodeI, b.nodeQ, R, b.small);
        g_launches += 1;
        l = b.deep_cut - 1;
    }
    auto *level = extra ? k_com_level<true> : k_com_level<false>;
    for (; l >= 1; --l) {
        level<<<grid, 256, 0, st>>>(l, b.nlist, b.spos, b.nodeW, b.nodeR, b.nodeD, b.nodeI,
                                    b.nodeQ, R, b.small);
        g_launches += 1;
    }
    if (b.nodeI) launch_root_moments(b, st);
}

void launch_root_moments(const BuildBufs &b, cudaStream_t st)
{
    k_root_moments<<<b.nsys, 32, 0, st>>>(b.sys, b.noff, b.spos, b.nodeW, b.nodeR, b.nodeD,
                                           b.nodeI, b.nodeQ, b.small);
    g_launches += 1;
}

void launch_sibling_order(const BuildBufs &b, cudaStream_t st)
{
    const uint32_t *mtot = b.noff + b.n_total;
    const int grid = b.nsm * 8;
    k_sib_count<<<grid, 256, 0, st>>>(mtot, b.node_cap, b.nodeW, b.nodeR, b.sib_count, b.small);
    launch_scan(b.sib_count, b.sib_count, (int)b.node_cap, b.scan_part, nullptr,
                &b.small->status, st);
    k_sib_place<<<grid, 256, 0, st>>>(mtot, b.nsys, b.nodeW, b.nodeR, b.sib_count, b.lidx,
                                      b.ldfs, b.small);
    k_sib_write<<<grid, 256, 0, st>>>(b.sys, b.noff, b.n_total, b.nodeW, b.nodeR, b.nodeD,
                                      b.lidx, b.ldfs, b.nodeF, b.nodeDF, b.small);
    g_launches += 3;
}

void launch_kick(const BuildBufs &b, cudaStream_t st)
{
    k_kick<<<b.nchunks, kWideThreads, 0, st>>>(b.chunks, b.sys, b.mode, b.small);
    g_launches += 1;
}

void launch_restore(const BuildBufs &b, cudaStream_t st)
{
    k_restore<<<b.nchunks, kWideThreads, 0, st>>>(b.chunks, b.sys, b.mode);
    g_launches += 1;
}

void launch_validate(const BuildBufs &b, cudaStream_t st)
{
    k_validate<<<b.nchunks, kChunkThreads, 0, st>>>(b.chunks, b.sys, b.small);
    g_launches += 1;
}

void launch_validate_arrays(const float4 *pos, const float4 *vel, int n, Small *sm, int nsm,
                            cudaStream_t st)
{
    k_validate_arrays<<<nsm * 4, 256, 0, st>>>(pos, vel, n, sm);
    g_launches += 1;
}

void launch_diagnostics(const BuildBufs &b, DiagPart *parts, double *out, cudaStream_t st)
{
    k_diag_part<<<b.nchunks, kChunkThreads, 0, st>>>(b.chunks, b.sys, parts);
    k_diag_final<<<b.nsys, 32, 0, st>>>(b.sys, parts, out);
    g_launches += 2;
}

void launch_export(const BuildBufs &b, int sysid, bh_node *nodes_dev, float4 *com_dev,
                   uint32_t *order_dev, cudaStream_t st)
{
    k_export<<<b.nsm * 4, 256, 0, st>>>(sysid, b.sys, b.noff, b.key0, b.val0, b.nodeW, b.nodeR,
                                        nodes_dev, com_dev, order_dev);
    g_launches += 1;
}

}  // namespace bh
