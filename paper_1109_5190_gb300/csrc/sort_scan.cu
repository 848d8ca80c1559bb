// sort_scan.cu -- segmented LSD radix sort of (63-bit Morton key, 32-bit id)
// pairs and a device-wide exclusive scan.
//
// The sort orders each system's particles by key; it is stable, and keys
// are produced in input order, so equal keys (coincident points at the depth
// cap) end up ordered by input index.  Eight passes of 8 bits each (or only the
// top few, then a fixup of short runs: see k_rs_fixup); every pass is
// histogram -> exclusive scan -> stable scatter.  Segmentation costs
// nothing extra: the per-(chunk, digit) counts are laid out system by system
// as [system][digit][chunk], so one global exclusive scan yields offsets that
// already include every earlier system's particles (chunks never straddle
// systems).  Only the first pass has a histogram kernel: each scatter also
// counts the next pass's digits per destination chunk.  Within a block, ranks come from warp-level __match_any_sync
// groups: one leader per digit and round updates the warp's running count,
// so no shared-memory atomics are needed and the order is stable.
#include "bh.h"
#include "bh_internal.cuh"

namespace bh {
namespace {

constexpr unsigned FULL = 0xffffffffu;
// Sort blocks: one chunk of kChunk keys per block of kSortThreads threads;
// warp w ranks elements [w * kPerWarp, (w + 1) * kPerWarp) in kRounds rounds.
constexpr int kSortThreads = 1024;
constexpr int kWarps = kSortThreads / 32;         // 32
constexpr int kPerWarp = kChunk / kWarps;         // 128
constexpr int kRounds = kPerWarp / 32;            // 4

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ unsigned count_index(const SysStatic &S, int chunk, int digit)
{
    return (unsigned)(kRadixBins * S.chunk0 + digit * S.nchunk + (chunk - S.chunk0));
}

__global__ void __launch_bounds__(kSortThreads)
k_rs_hist(const uint64_t *__restrict__ key, const int4 *__restrict__ chunks,
          const SysStatic *__restrict__ sys, uint32_t *__restrict__ counts, int shift,
          const Small *__restrict__ sm)
{
    if (sm->status) return;
    __shared__ uint32_t h[kWarps][kRadixBins];
    for (int q = threadIdx.x; q < kWarps * kRadixBins; q += blockDim.x) (&h[0][0])[q] = 0;
    __syncthreads();
    const int4 c = chunks[blockIdx.x];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int r = 0; r < kRounds; ++r) {
        const int i = w * kPerWarp + r * 32 + lane;
        const bool valid = i < c.z;
        const unsigned d = valid ? (unsigned)((key[c.y + i] >> shift) & (kRadixBins - 1)) : kRadixBins;
        const unsigned peers = __match_any_sync(FULL, d);
        if (valid && (peers & lanemask_lt()) == 0) h[w][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    const SysStatic S = sys[c.x];
    for (int d = threadIdx.x; d < kRadixBins; d += blockDim.x) {
        uint32_t t = 0;
        for (int q = 0; q < kWarps; ++q) t += h[q][d];
        counts[count_index(S, blockIdx.x, d)] = t;
    }
}

constexpr int kScanThreads = 256;
constexpr int kScanItems = kScanTile / kScanThreads;  // 8

// Exclusive scan of the block's values (one per thread); returns the
// exclusive prefix and writes the block total to *total.
__device__ __forceinline__ uint32_t block_exclusive(uint32_t x, uint32_t *total)
{
    __shared__ uint32_t ws[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = x;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) ws[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t s = lane < nw ? ws[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, s, o);
            if (lane >= o) s += y;
        }
        ws[lane] = s;  // inclusive over warps
    }
    __syncthreads();
    const uint32_t wbase = w ? ws[w - 1] : 0u;
    const uint32_t tot = ws[nw - 1];
    __syncthreads();
    *total = tot;
    return wbase + inc - x;
}

// Scatter of one chunk: ranks as in the histogram (stable), then the chunk is
// laid out in digit order in shared memory and written from there, so
// neighbouring threads write neighbouring addresses of one digit's run
// (coalesced), and the next pass's digits are counted per destination chunk.
// Dynamic shared memory: per-warp counts | global bases | block bases | keys | ids.
constexpr size_t kScatterSmem = sizeof(uint32_t) * (kWarps * kRadixBins + 2 * kRadixBins) +
                                sizeof(uint64_t) * kChunk + sizeof(uint32_t) * kChunk;

__global__ void __launch_bounds__(kSortThreads, 2)
k_rs_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
             uint64_t *__restrict__ kout, uint32_t *__restrict__ vout,
             const int4 *__restrict__ chunks, const SysStatic *__restrict__ sys,
             const uint32_t *__restrict__ offs, int shift, uint32_t *__restrict__ next_counts,
             const Small *__restrict__ sm)
{
    if (sm->status) return;
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t(*h)[kRadixBins] = reinterpret_cast<uint32_t(*)[kRadixBins]>(smem);
    uint32_t *gbase = reinterpret_cast<uint32_t *>(smem) + kWarps * kRadixBins;
    uint32_t *bstart = gbase + kRadixBins;
    uint64_t *skey = reinterpret_cast<uint64_t *>(bstart + kRadixBins);
    uint32_t *sval = reinterpret_cast<uint32_t *>(skey + kChunk);
    for (int q = threadIdx.x; q < kWarps * kRadixBins; q += blockDim.x) (&h[0][0])[q] = 0;
    __syncthreads();
    const int4 c = chunks[blockIdx.x];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    // only (rank, digit) stays in registers between the two phases; keys and
    // ids are read again (L2 hits) when staged: the block runs at 32
    // registers per thread, and holding them would spill to local memory
    uint32_t rd[kRounds];  // (rank within warp << 9) | digit (digit 256 = empty slot)
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const int i = w * kPerWarp + r * 32 + lane;
        const bool valid = i < c.z;
        unsigned d = kRadixBins;
        if (valid) d = (unsigned)((kin[c.y + i] >> shift) & (kRadixBins - 1));
        const unsigned peers = __match_any_sync(FULL, d);
        const unsigned before = valid ? h[w][d] : 0u;
        __syncwarp();
        if (valid && (peers & lt) == 0) h[w][d] = before + __popc(peers);
        __syncwarp();
        rd[r] = ((before + __popc(peers & lt)) << 9) | d;
    }
    __syncthreads();
    const SysStatic S = sys[c.x];
    uint32_t total = 0;
    if (threadIdx.x < kRadixBins) {
        const int d = threadIdx.x;
        for (int q = 0; q < kWarps; ++q) {
            const uint32_t t = h[q][d];
            h[q][d] = total;
            total += t;
        }
        gbase[d] = offs[count_index(S, blockIdx.x, d)];
    }
    uint32_t dummy;
    const uint32_t bs = block_exclusive(threadIdx.x < kRadixBins ? total : 0u, &dummy);
    if (threadIdx.x < kRadixBins) bstart[threadIdx.x] = bs;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const unsigned d = rd[r] & 511u;
        if (d < (unsigned)kRadixBins) {
            const int i = w * kPerWarp + r * 32 + lane;
            const uint32_t p = bstart[d] + h[w][d] + (rd[r] >> 9);
            skey[p] = kin[c.y + i];
            sval[p] = vin[c.y + i];
        }
    }
    __syncthreads();
    for (int q0 = 0; q0 < kChunk; q0 += kSortThreads) {
        const int q = q0 + threadIdx.x;
        const bool valid = q < c.z;
        uint32_t dst = 0;
        uint64_t key = 0;
        if (valid) {
            key = skey[q];
            const unsigned d = (unsigned)((key >> shift) & (kRadixBins - 1));
            dst = gbase[d] + ((uint32_t)q - bstart[d]);
            kout[dst] = key;
            vout[dst] = sval[q];
        }
        if (next_counts) {
            // the next pass's histogram: count this key's next digit in the
            // chunk it lands in (warp-aggregated global atomics)
            unsigned idx = 0xffffffffu;
            if (valid) {
                const int chunk = S.chunk0 + ((int)dst - S.start) / kChunk;
                const int nd = (int)((key >> (shift + kRadixBits)) & (kRadixBins - 1));
                idx = count_index(S, chunk, nd);
            }
            const unsigned peers = __match_any_sync(FULL, idx);
            if (valid && (peers & lt) == 0) atomicAdd(&next_counts[idx], (unsigned)__popc(peers));
        }
    }
}

// ---------------------------------------------------------------- scan

// Tile sums part[b] of the input; also clears zero[0..nzero) (the next
// radix pass's count buffer), which saves the stream a separate memset.
__global__ void __launch_bounds__(kScanThreads)
k_scan_reduce(const uint32_t *__restrict__ in, int n, uint32_t *__restrict__ part,
              uint32_t *__restrict__ zero, int nzero, const int *__restrict__ status)
{
    if (status && *status) return;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nzero; q += gridDim.x * blockDim.x)
        zero[q] = 0u;
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q)
        if (base + q < n) s += in[base + q];
    uint32_t tot;
    block_exclusive(s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// Scans part[0..nb) in place (exclusive); *total = sum.  Used when there are
// more tiles than k_scan_apply adds up inline.
__global__ void __launch_bounds__(1024)
k_scan_part(uint32_t *__restrict__ part, int nb, uint32_t *__restrict__ total,
            const int *__restrict__ status)
{
    if (status && *status) return;
    uint32_t carry = 0;
    for (int b0 = 0; b0 < nb; b0 += 1024 * 4) {
        const int base = b0 + threadIdx.x * 4;
        uint32_t x[4], s = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            x[q] = (base + q < nb) ? part[base + q] : 0u;
            s += x[q];
        }
        uint32_t tot;
        uint32_t e = block_exclusive(s, &tot) + carry;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (base + q < nb) part[base + q] = e;
            e += x[q];
        }
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

// Up to this many tiles, each k_scan_apply block adds up the tile sums before
// its own (one load per thread), so no separate pass scans them.
constexpr int kScanInlineTiles = kScanThreads;

// Scans tile b.  inline_part: part[] holds raw tile sums and the block adds
// up those before it, and the last block writes the grand total to *total
// (if given); otherwise part[] was scanned by k_scan_part.
__global__ void __launch_bounds__(kScanThreads)
k_scan_apply(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, int n,
             const uint32_t *__restrict__ part, int inline_part, uint32_t *__restrict__ total,
             const int *__restrict__ status)
{
    if (status && *status) return;
    uint32_t offset;
    if (inline_part) {
        uint32_t before = 0;
        for (int q = threadIdx.x; q < (int)blockIdx.x; q += blockDim.x) before += part[q];
        block_exclusive(before, &offset);
    } else {
        offset = part[blockIdx.x];
    }
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    uint32_t x[kScanItems], s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        x[q] = (base + q < n) ? in[base + q] : 0u;
        s += x[q];
    }
    uint32_t tot;
    uint32_t e = block_exclusive(s, &tot) + offset;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        if (base + q < n) out[base + q] = e;
        e += x[q];
    }
    if (inline_part && total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
        *total = offset + tot;
}

// One block scans up to kScanSingleMax values: rows of 4096 (4 per thread,
// contiguous, so loads coalesce) with a running carry.
constexpr int kScanSingleMax = 8192;

__global__ void __launch_bounds__(1024)
k_scan_single(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, int n,
              uint32_t *__restrict__ total, const int *__restrict__ status)
{
    if (status && *status) return;
    uint32_t carry = 0;
    for (int b0 = 0; b0 < n; b0 += 1024 * 4) {
        const int base = b0 + threadIdx.x * 4;
        uint32_t x[4], s = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            x[q] = (base + q < n) ? in[base + q] : 0u;
            s += x[q];
        }
        uint32_t tot;
        uint32_t e = block_exclusive(s, &tot) + carry;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (base + q < n) out[base + q] = e;
            e += x[q];
        }
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

}  // namespace

namespace {

// launch_scan, and also clears zero[0..nzero) on the way
void scan_and_clear(const uint32_t *in, uint32_t *out, int n, uint32_t *partials,
                    uint32_t *total, const int *status, cudaStream_t st, uint32_t *zero,
                    int nzero)
{
    if (n <= 0) return;
    if (n <= kScanSingleMax) {
        if (nzero > 0) cudaMemsetAsync(zero, 0, sizeof(uint32_t) * (size_t)nzero, st);
        k_scan_single<<<1, 1024, 0, st>>>(in, out, n, total, status);
        g_launches += 1;
        return;
    }
    const int nb = (n + kScanTile - 1) / kScanTile;
    const int inline_part = nb <= kScanInlineTiles;
    k_scan_reduce<<<nb, kScanThreads, 0, st>>>(in, n, partials, zero, nzero, status);
    if (!inline_part) {
        k_scan_part<<<1, 1024, 0, st>>>(partials, nb, total, status);
        g_launches += 1;
    }
    k_scan_apply<<<nb, kScanThreads, 0, st>>>(in, out, n, partials, inline_part, total, status);
    g_launches += 2;
}

}  // namespace

void launch_scan(const uint32_t *in, uint32_t *out, int n, uint32_t *partials, uint32_t *total,
                 const int *status, cudaStream_t st)
{
    scan_and_clear(in, out, n, partials, total, status, st, nullptr, 0);
}

// Opts the scatter in to more than 48 KiB of dynamic shared memory; called
// once per context before any launch (and so before any stream capture).
void prepare_sort_kernels()
{
    cudaFuncSetAttribute(k_rs_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kScatterSmem);
}

// The short sort: LSD passes over the top digits only (passes first..7, key
// bits 8 * first..63), so the keys end up ordered by those bits, ties in input
// order.  A run of keys equal there (particles sharing a cell of about level
// (63 - 8 * first) / 3) is then put in order by its full key, stably, which
// gives exactly the (key, input index) order of the full sort.  The fixup
// writes the result to the first buffers (from the second after an odd
// number of passes).
constexpr int kRunMax = 8;

__global__ void __launch_bounds__(kWideThreads)
k_rs_fixup(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
           uint64_t *__restrict__ kout, uint32_t *__restrict__ vout,
           const int4 *__restrict__ chunks, const SysStatic *__restrict__ sys, int kTopShift,
           Small *__restrict__ sm)
{
    if (sm->status) return;
    const int4 c = chunks[blockIdx.x];
    const SysStatic S = sys[c.x];
    const int send = S.start + S.n;
    for (int k = 0; k < kWideItems; ++k) {
        const int i = k * kWideThreads + threadIdx.x;
        if (i >= c.z) break;
        const int j = c.y + i;
        const uint64_t kj = kin[j];
        const uint64_t pj = kj >> kTopShift;
        // a run is written by the thread of its first key
        if (j > S.start && (kin[j - 1] >> kTopShift) == pj) continue;
        int len = 1;
        while (len <= kRunMax && j + len < send && (kin[j + len] >> kTopShift) == pj) ++len;
        if (len > kRunMax) {
            atomicExch(&sm->status, ST_SORT_LONG);
            continue;
        }
        if (len == 1) {
            kout[j] = kj;
            vout[j] = vin[j];
            continue;
        }
        uint64_t rk[kRunMax];
        uint32_t rv[kRunMax];
        for (int q = 0; q < len; ++q) {
            rk[q] = kin[j + q];
            rv[q] = vin[j + q];
        }
        // insertion sort, stable: an element moves only past larger keys
        for (int q = 1; q < len; ++q) {
            const uint64_t x = rk[q];
            const uint32_t y = rv[q];
            int p = q;
            while (p > 0 && rk[p - 1] > x) {
                rk[p] = rk[p - 1];
                rv[p] = rv[p - 1];
                --p;
            }
            rk[p] = x;
            rv[p] = y;
        }
        for (int q = 0; q < len; ++q) {
            kout[j + q] = rk[q];
            vout[j + q] = rv[q];
        }
    }
}

void launch_sort(const BuildBufs &b, cudaStream_t st)
{
    uint64_t *kin = b.key0, *kout = b.key1;
    uint32_t *vin = b.val0, *vout = b.val1;
    const int ncounts = kRadixBins * b.nchunks;
    // two count buffers: pass p scans and reads one while its scatter counts
    // the next pass's digits into the other (zeroed just before)
    uint32_t *cur = b.rs_counts, *nxt = b.rs_counts + ncounts;
    const int first = b.sort_first;
    k_rs_hist<<<b.nchunks, kSortThreads, 0, st>>>(kin, b.chunks, b.sys, cur, first * kRadixBits,
                                                  b.small);
    g_launches += 1;
    for (int pass = first; pass < kRadixPasses; ++pass) {
        const int shift = pass * kRadixBits;
        const bool more = pass + 1 < kRadixPasses;
        // the scan also clears the count buffer this pass's scatter fills
        scan_and_clear(cur, cur, ncounts, b.scan_part, nullptr, &b.small->status, st, nxt,
                       more ? ncounts : 0);
        k_rs_scatter<<<b.nchunks, kSortThreads, kScatterSmem, st>>>(
            kin, vin, kout, vout, b.chunks, b.sys, cur, shift, more ? nxt : nullptr, b.small);
        g_launches += 1;
        uint64_t *tk = kin; kin = kout; kout = tk;
        uint32_t *tv = vin; vin = vout; vout = tv;
        uint32_t *tc = cur; cur = nxt; nxt = tc;
    }
    if (first > 0) {  // the keys are in kin: the second buffers after an odd pass count
        k_rs_fixup<<<b.nchunks, kWideThreads, 0, st>>>(kin, vin, b.key0, b.val0, b.chunks, b.sys,
                                                       first * kRadixBits, b.small);
        g_launches += 1;
    }
}

}  // namespace bh
