// bh_internal.cuh -- device data layout and kernel launchers shared by the
// library's translation units.  Not part of the public ABI (see include/bh.h).
//
// Layout in HBM (one "forest" = one or more independent systems):
//   * Per system, in the caller's particle order: pos (x,y,z,m), vel, acc
//     (ax,ay,az,phi) as float4 arrays, plus a backup of pos/vel taken at the
//     start of every step (used to roll a step back after a node-buffer
//     overflow).
//   * Systems are concatenated in a "virtual" index space [0, n_total);
//     system s owns [start_s, start_s + n_s).  Every O(n) kernel runs over
//     chunks of <= kChunk particles that never straddle two systems, so a
//     block finds its system with one table lookup.
//   * Sorted working arrays in virtual index space: 64-bit keys and 32-bit
//     virtual ids (double-buffered for the radix sort), the Morton-ordered
//     copy spos of pos_mass, per-particle node counts / offsets.
//   * Nodes of all trees in one array, each system's nodes contiguous, in
//     depth-first pre-order (the canonical order): the 32-byte walk record
//     WNode (below), the rarely used fields nodeR = (first, count, level, 0)
//     and the FP64 centre of mass nodeD = (mass, cx, cy, cz), which the
//     bottom-up pass works in and the walk reads only to re-decide opening
//     tests that fall within rounding distance of a tie.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace bh {

constexpr int kLevels = BH_MAX_DEPTH;  // 21
constexpr int kNumLevels = kLevels + 1;
constexpr int kChunk = 4096;
constexpr int kChunkThreads = 256;
constexpr int kItems = kChunk / kChunkThreads;  // 16
// kernels whose per-particle work is a chain of dependent loads (topology,
// keys, permutation, closing kick) run more threads per chunk, each with fewer
// particles; those that end in a block reduction keep kChunkThreads
constexpr int kWideThreads = 1024;
constexpr int kWideItems = kChunk / kWideThreads;  // 4
constexpr float kLeafCrit = -1.0f;
constexpr float kBucketCrit = __builtin_huge_valf();  // +inf: never accepted as a whole
constexpr int kRadixBits = 8;
constexpr int kRadixBins = 1 << kRadixBits;
constexpr int kRadixPasses = 8;  // 63-bit keys
constexpr int kScanTile = 2048;
// relative half-width of the band around an opening threshold inside which
// the FP32 test is re-decided in FP64
constexpr float kTieBand = 4e-6f;

// device status codes (0 = ok)
// ST_SORT_LONG: the short sort met a run of more than kRunMax keys equal in
// their sorted top digits; the step is redone with one digit more
enum : int { ST_OK = 0, ST_CAPACITY = 1, ST_WALK_LIMIT = 2, ST_BAD_INPUT = 3, ST_SORT_LONG = 4 };

// per-system modes of one step
enum : int { MODE_ACCEL = 0, MODE_KDK = 1, MODE_IDLE = 2 };

struct SysStatic {
    float4 *pos, *vel, *acc, *bpos, *bvel;
    int start, n;
    int chunk0, nchunk;
    float eps2, G, inv_theta2, half_dt;
    float dt;
    int flags;
    double theta2;
};

struct SysDyn {
    float lo[3];
    float side;
    float scale;
    float root_m;
    float root_com[3];
    float pad;
    double mtot;
    double mx[3];
};

struct ChunkPart {
    float mn[3];
    float mx[3];
    float pad[2];
    double m, sx, sy, sz;
};

struct DiagPart {
    double v[9];  // KE, PE, Px, Py, Pz, M, Mx, My, Mz
    double pad;
};

constexpr int kMaxTileGroups = 256;  // SMs whose walk tiles are shared per SM

// Small per-forest device scalars.  The block [queue .. level_cur] is zeroed
// at the start of every step with one memset.
struct Small {
    int status;
    unsigned M;
    unsigned needed;
    unsigned steps_done;
    // counting walk: interactions, warp iterations, particle-slot node visits
    unsigned long long wstats[3];
    unsigned queue;
    unsigned ranges_empty;  // the walk's per-SM tile ranges found empty
    // the walk's per-SM tile ranges: tiles taken from the front (low 32 bits,
    // by the SM's own warps) and from the back (high 32 bits, by other SMs')
    unsigned long long group_ctr[kMaxTileGroups];
    unsigned level_cnt[kNumLevels];
    unsigned level_cur[kNumLevels];
    unsigned level_off[kNumLevels + 1];
};

// The walk's node record: 32 bytes, one DRAM/L2 sector.
//   a = (hx, hy, hz, mass)   FP32 centre of mass (high part) and mass
//   b = (crit2 bits, skip, lo_xy, lo_z | e << 23)
//       crit2 = s^2/theta^2 (accept iff d^2 > crit2), -1 for a one-particle
//       leaf (always taken as is), +inf for a depth-cap bucket (never taken
//       as a whole: its particles are summed one by one); skip = index of
//       the next node after the subtree (> the node's own index); the low part com - h of each
//       coordinate as an int16 multiple of 2^(e - 127) (e chosen per node
//       from the largest |h|, so the low part keeps 2^-16 of an FP32 ulp).
// Fields the walk rarely needs live in nodeR = (first, count, level, system).
struct __align__(32) WNode {
    float4 a;
    uint4 b;
};

// Sibling-order copy of the records (walk shape BH_GROUP_SIBLINGS): system s's
// root at index s, then the children of every node next to each other, the
// blocks in the depth-first order of their parents.  The walk gets these
// records as WalkArgs::nodeW and a sibling-order copy of the FP64 centres of
// mass as WalkArgs::nodeD.
// Same 32 bytes, same a, lo parts and exponent; b differs:
//   b = (target, next, lo_xy, lo_z | level << 16 | kind << 21 | e << 23)
//   kind kSibCell: target = sibling-order index of the first child; the
//       threshold is s^2/theta^2 from the level, as the topology pass forms it;
//   kind kSibLeaf: target = the particle (sorted index);
//   kind kSibBucket (a depth-cap bucket, or any cell when theta = 0):
//       target = the node's depth-first index (its members are in nodeR);
//   next = sibling-order index of the node after the subtree in depth-first
//       order, or kSibEnd after the system's last node.
constexpr unsigned kSibCell = 0, kSibLeaf = 1, kSibBucket = 2;
constexpr unsigned kSibEnd = 0xffffffffu;

#ifdef __CUDACC__
__device__ __forceinline__ float wn_crit(const uint4 &b) { return __uint_as_float(b.x); }
__device__ __forceinline__ int wn_skip(const uint4 &b) { return (int)b.y; }

__device__ __forceinline__ void wn_lo(const uint4 &b, float &lx, float &ly, float &lz)
{
    const float scale = __int_as_float(b.w & 0x7f800000u);
    lx = (float)(short)(b.z & 0xffffu) * scale;
    ly = (float)(short)(b.z >> 16) * scale;
    lz = (float)(short)(b.w & 0xffffu) * scale;
}

// Packs threshold, skip pointer and the low parts com - h (FP64) of a node.
__device__ __forceinline__ uint4 wn_pack(float crit, int skip, double cx, double cy, double cz,
                                         float hx, float hy, float hz)
{
    const float mx = fmaxf(fabsf(hx), fmaxf(fabsf(hy), fabsf(hz)));
    // |com - h| <= ulp(mx)/2 = 2^(E-151); the scale 2^(E-165) keeps |q| <= 2^14
    int e = ((__float_as_int(mx) >> 23) & 0xff) - 38;
    if (e < 1) e = 1;
    const double inv = __longlong_as_double((long long)(1023 - (e - 127)) << 52);
    const int qx = max(-32767, min(32767, __double2int_rn((cx - (double)hx) * inv)));
    const int qy = max(-32767, min(32767, __double2int_rn((cy - (double)hy) * inv)));
    const int qz = max(-32767, min(32767, __double2int_rn((cz - (double)hz) * inv)));
    return make_uint4(__float_as_uint(crit), (unsigned)skip,
                      ((unsigned)qx & 0xffffu) | ((unsigned)qy << 16),
                      ((unsigned)qz & 0xffffu) | ((unsigned)e << 23));
}
#endif

struct Tile {
    int start;  // virtual index of the first particle (sorted order)
    int count;  // <= 32 * ppl
    int sys;
    int pad;
};

// ------------------------------------------------------------- launchers

struct BuildBufs {
    const int4 *chunks;  // (sys, start, count, 0)
    int nchunks;
    const SysStatic *sys;
    SysDyn *dyn;
    int nsys;
    const int *mode;  // per system
    ChunkPart *parts;
    uint64_t *key0, *key1;
    uint32_t *val0, *val1;
    uint32_t *rs_counts;  // kRadixBins * nchunks
    // first radix pass: 0 = all eight digits; k > 0 = passes k..7 only (the
    // top 8 - k digits), then each run of keys equal there is put in order
    // (ST_SORT_LONG if a run is longer than kRunMax)
    int sort_first;
    uint32_t *scan_part;  // scan partials
    float4 *spos;
    uint32_t *ncount;     // n_total + 1
    uint32_t *noff;       // n_total + 1
    WNode *nodeW;
    int4 *nodeR;
    double4_32a *nodeD;
    uint32_t *nlist;
    // quadrupole mode only (else null): FP64 second moments about the centre
    // of mass (xx, yy, zz, xy, xz, yz per node) and their FP32 copy for the
    // walk, two float4 per node: (xx, yy, zz, xy), (xz, yz, 0, 0)
    double *nodeI;
    float4 *nodeQ;
    // b_max rule only (else null): FP64 b_max^2 per cell, the size that the
    // rule puts in the opening test in place of the side
    double *nodeB;
    // sibling-order walk only (else null): the sibling-order records and FP64
    // centres of mass, the maps depth-first -> sibling order (lidx) and back
    // (ldfs), and per-node child counts (node_cap entries, scanned in place)
    WNode *nodeF;
    double4_32a *nodeDF;
    uint32_t *lidx, *ldfs, *sib_count;
    unsigned node_cap;
    Small *small;
    int n_total;
    int nsm;
    // levels deep_cut .. 21 hold few nodes: their centres of mass are done in
    // one single-block launch (22 = none); any value gives the same result
    int deep_cut;
};

void launch_kick_drift_bbox(const BuildBufs &b, cudaStream_t st);
void launch_keys(const BuildBufs &b, cudaStream_t st);
void launch_sort(const BuildBufs &b, cudaStream_t st);
void prepare_sort_kernels();
void launch_permute(const BuildBufs &b, cudaStream_t st);
void launch_topology(const BuildBufs &b, cudaStream_t st);
void launch_com(const BuildBufs &b, cudaStream_t st);
void launch_root_moments(const BuildBufs &b, cudaStream_t st);  // quadrupole mode
void launch_sibling_order(const BuildBufs &b, cudaStream_t st);  // sibling-order walk
void launch_kick(const BuildBufs &b, cudaStream_t st);
void launch_restore(const BuildBufs &b, cudaStream_t st);
void launch_validate(const BuildBufs &b, cudaStream_t st);
void launch_validate_arrays(const float4 *pos, const float4 *vel, int n, Small *sm, int nsm,
                            cudaStream_t st);
void launch_diagnostics(const BuildBufs &b, DiagPart *parts, double *out, cudaStream_t st);
void launch_export(const BuildBufs &b, int sys, bh_node *nodes_dev, float4 *com_dev,
                   uint32_t *order_dev, cudaStream_t st);

// generic exclusive scan of n uint32 (out may alias in); total -> *total
void launch_scan(const uint32_t *in, uint32_t *out, int n, uint32_t *partials,
                 uint32_t *total, const int *status, cudaStream_t st);

struct WalkArgs {
    const WNode *nodeW;
    const float4 *nodeQ;  // quadrupole mode: 2 float4 per node (else null)
    const int4 *nodeR;
    const double4_32a *nodeD;
    const double *nodeB;  // b_max rule: FP64 b_max^2 per cell (else null)
    const SysDyn *dyn;
    const float4 *spos;
    const uint32_t *sid;  // sorted -> virtual id
    const uint32_t *noff;
    const Tile *tiles;
    int ntiles;
    const SysStatic *sys;
    const int *mode;
    Small *small;
    uint32_t *counts;  // per-particle interaction counts (virtual order) or null
    int static_share;  // percent of tiles split into per-SM contiguous ranges (with stealing)
    int nsm;           // SMs the persistent grid is spread over
};

// ppl: particles per lane; group: lanes that vote together on the next node
// (32 = the whole warp walks the union of its particles' traversals, 1 =
// every lane walks its own particles' traversal independently)
struct WalkShape {
    int ppl;
    int warps;
    int blocks_per_sm;
    int group;
    bool open_inside;  // BH_OPEN_INSIDE: one particle per lane, group 1
    bool quad;         // BH_QUADRUPOLE: one particle per lane, group 1, Kahan
    bool soft;         // every system has eps > 0 (no zero-distance guard needed)
};

// kahan / potential / counting variants; returns number of kernel launches
int launch_walk(const WalkArgs &a, const WalkShape &sh, bool kahan, bool pot, bool count,
                int nsm, cudaStream_t st);
int walk_max_blocks_per_sm(const WalkShape &sh, bool kahan, bool pot);

// micro-benchmarks
double micro_fma_gflops(cudaStream_t st);
double micro_l1_sectors(cudaStream_t st);  // G sectors/s of scattered 32-byte L1 loads
double micro_copy_gbs(size_t bytes, cudaStream_t st);

// number of kernel launches issued by the last launch_* helper call on
// this thread (used for the launch count reported by profiling)
extern thread_local int g_launches;

}  // namespace bh
