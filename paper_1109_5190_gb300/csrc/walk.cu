// walk.cu -- the Barnes-Hut force walk: the per-particle force phase, which
// Section III names as the costliest phase of the method.
//
// For each particle i the walk sums, over the cells it accepts and the leaf
// particles it reaches, G m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^(3/2).  A
// cell of side s at distance d (to its centre of mass) is accepted iff
// s^2 < theta^2 d^2 (Section III, Fig. 1, with r the cell side); otherwise
// its children are visited.  The decision is taken per particle, exactly.
//
// GPU design (sm_103a; bound by L1's data pipe for the scattered node loads,
// not by FP32 math; no tensor cores: this is not a dense contraction):
//   * Persistent kernel; each warp pulls tiles of 32*PPL consecutive
//     Morton-sorted particles: first from its SM's contiguous share of a
//     tunable fraction of the tiles (neighbouring walks share L1), then from
//     an atomic queue over the rest (dynamic load balancing in place of the
//     paper's runtime work queues, Section III).
//   * Stackless traversal: nodes are stored in depth-first pre-order with a
//     skip pointer (the first node after the subtree).  Each particle slot
//     keeps the index of the next node it must visit (the root at first);
//     accepting continues at the skip pointer, opening at the next node (the
//     first child).
//   * Lanes vote on the next node in aligned groups of GROUP lanes.  GROUP 1:
//     no vote, every lane walks its own particle (the usual choice: the lanes
//     of a tile start together and share most node loads).  GROUP 32: the
//     warp takes the smallest next index (__reduce_min_sync), reads that node
//     once for all lanes, and every slot waiting on it decides for itself --
//     the union of the tile's walks.  The vote replaces an explicit per-warp
//     (node, lane-mask) stack: the slots waiting on a node are exactly the
//     mask such a stack would carry, and no stack can overflow.
//   * k_walk_split (below) votes over the top levels only and walks the rest
//     lane by lane.
//   * One-particle leaves carry threshold -1 (always accepted as the particle
//     itself); depth-cap buckets carry +inf (never accepted as a whole) and
//     are summed particle by particle where a walk would open them.
//   * Compensated (Kahan) FP32 accumulation of each force component (and of
//     the potential when requested).
//   * The loop's trip count is bounded by the node count: every iteration
//     strictly increases the smallest next index, because every skip pointer
//     lies past its node.  The topology pass checks that for each node it
//     writes (index < skip <= end of the system's nodes); a violation is a
//     corrupt tree: it sets ST_WALK_LIMIT and no later kernel, the walk
//     included, runs.
#include <algorithm>
#include <atomic>

#include "bh.h"
#include "bh_internal.cuh"

namespace bh {
namespace {

constexpr unsigned FULL = 0xffffffffu;

// The whole 32-byte node record in one 256-bit read-only load.
__device__ __forceinline__ void load_node(const WNode *p, float4 &A, uint4 &B)
{
    float b0, b1, b2, b3;
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(A.x), "=f"(A.y), "=f"(A.z), "=f"(A.w), "=f"(b0), "=f"(b1), "=f"(b2), "=f"(b3)
        : "l"(p));
    B = make_uint4(__float_as_uint(b0), __float_as_uint(b1), __float_as_uint(b2), __float_as_uint(b3));
}

template <bool KAHAN>
__device__ __forceinline__ void acc_add(float &s, float &c, float x)
{
    if (KAHAN) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    } else {
        s += x;
    }
}

// s += a * b, compensated: the term's product and the correction carried from
// the previous step are taken in one fused multiply-add.
template <bool KAHAN>
__device__ __forceinline__ void acc_fma(float &s, float &c, float a, float b)
{
    if (KAHAN) {
        const float y = fmaf(a, b, -c);
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    } else {
        s = fmaf(a, b, s);
    }
}

// The opening test s^2 < theta^2 d^2 as the walk first takes it, in FP32 on
// the node's stored threshold crit = s^2 / theta^2: accept when d^2 exceeds
// crit by more than the relative tie band, open when it falls short of it by
// more; a test inside the band is re-decided in FP64 (accept_fp64).  Each
// bound is one fused multiply-add with one rounding, so its sign is that of
// the exact difference.  Leaves (crit = -1) are always accepted; buckets and
// theta = 0 (crit = +inf) always open, without an FP64 test.
__device__ __forceinline__ bool fp32_accepts(float d2, float crit)
{
    return fmaf(-crit, 1.0f + kTieBand, d2) > 0.f;
}
__device__ __forceinline__ bool fp32_opens(float d2, float crit)
{
    return fmaf(-crit, 1.0f - kTieBand, d2) < 0.f;
}

// The paper's opening test in FP64, for a test whose FP32 value lies within
// rounding distance of the threshold: s^2 < theta^2 d^2 with s = side 2^-level
// and d from the FP64 centre of mass (the same formula and operation order as
// the FP64 definition, so both decide alike).
// Out of line on purpose: the rare FP64 path then keeps its registers (and
// its FP64 arithmetic) out of the walk loop.
__device__ __noinline__ bool accept_fp64(const double4_32a *__restrict__ nodeD,
                                         const int4 *__restrict__ nodeR,
                                         const double *__restrict__ nodeB,
                                         const SysStatic *__restrict__ sys,
                                         const SysDyn *__restrict__ dyn, int sysid, int node,
                                         float px, float py, float pz)
{
    const double theta2 = sys[sysid].theta2;
    const double4_32a D = nodeD[node];
    const double dx = __dsub_rn(D.y, (double)px);
    const double dy = __dsub_rn(D.z, (double)py);
    const double dz = __dsub_rn(D.w, (double)pz);
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    double r2;  // the cell's size squared: b_max^2 under the b_max rule, else s^2
    if (nodeB) {
        r2 = nodeB[node];
    } else {
        const double s = (double)dyn[sysid].side *
                         __longlong_as_double((long long)(1023 - nodeR[node].z) << 52);
        r2 = __dmul_rn(s, s);
    }
    return r2 < __dmul_rn(theta2, d2);
}

// Offset within its tile of a lane's k-th particle.  When the whole warp
// votes (GROUP 32) every lane sees the union anyway, so slot k of all lanes is
// one contiguous run of 32; with smaller vote groups a lane's own particles
// are neighbours in Morton order, so their traversals nearly coincide and one
// node load serves all of them.
template <int PPL, int GROUP>
__device__ __forceinline__ int slot_offset(int lane, int k)
{
    return GROUP == 32 ? k * 32 + lane : lane * PPL + k;
}

// Hands out a walk's tiles.  Tiles [0, nstatic) (the static share) are split
// into one contiguous range per SM: the blocks on an SM (block b on SM
// b mod #SMs, the order a persistent grid is dealt in) take its tiles from the
// front through one counter in global memory, so all of the SM's warps walk
// neighbouring tiles and share tree nodes in L1.  A warp whose SM's range is
// empty takes single tiles from the back of the other SMs' ranges, nearest
// SMs first (their tiles are the nearest in Morton order), until every range
// is empty, which evens out the finishing times without scattering the tail.  The rest of the tiles go
// through a global atomic queue.  One 64-bit counter per range holds the
// tiles taken from the front (low 32 bits) and from the back (high 32 bits);
// a take is valid iff the two counts before it sum to less than the range's
// length, so every tile is taken exactly once.  Any other placement of blocks
// only shares less; a grid that is not #SMs x blocks-per-SM uses one range
// per block, counted in shared memory (s_next, zeroed by the caller before a
// block barrier), and no taking from other ranges.
struct TileDealer {
    unsigned long long *ctr;  // per-SM range counters (null: one range per block)
    unsigned *empty;          // ranges found empty so far
    unsigned *s_next;         // per-block range counter
    unsigned *queue;          // dynamic queue
    int group, ngroups, per_group, nstatic;
    // the taking warp's state (lane 0): its own range is empty; ranges tried
    bool own_done = false;
    int tried = 0;

    __device__ __forceinline__ TileDealer(const WalkArgs &a, unsigned *next_in_block)
    {
        const int bps = a.nsm > 0 ? (int)gridDim.x / a.nsm : 1;
        const bool per_sm = a.nsm > 0 && bps * a.nsm == (int)gridDim.x && a.nsm <= kMaxTileGroups;
        ngroups = per_sm ? a.nsm : (int)gridDim.x;
        group = per_sm ? (int)blockIdx.x % a.nsm : (int)blockIdx.x;
        ctr = per_sm ? a.small->group_ctr : nullptr;
        empty = &a.small->ranges_empty;
        s_next = next_in_block;
        queue = &a.small->queue;
        per_group = (int)(((long long)a.ntiles * a.static_share / 100) / ngroups);
        nstatic = per_group * ngroups;
    }

    // One take from range v (front: its own SM's warps; back: others').  The
    // take whose counts before it sum to exactly the range's length is the
    // first to find it empty, and counts it.
    __device__ __forceinline__ int take_from(int v, bool back) const
    {
        const unsigned long long o = atomicAdd(&ctr[v], back ? 1ull << 32 : 1ull);
        const int f = (int)(unsigned)o, b = (int)(o >> 32);
        if (f + b < per_group) return v * per_group + (back ? per_group - 1 - b : f);
        if (f + b == per_group) atomicAdd(empty, 1u);
        return -1;
    }

    // the warp's next tile (lane 0 takes it; every lane gets it)
    __device__ __forceinline__ int take(int lane)
    {
        int t = -1;
        if (lane == 0) {
            if (!ctr) {
                const int k = (int)atomicAdd(s_next, 1u);
                if (k < per_group) t = group * per_group + k;
            } else {
                if (!own_done) {
                    t = take_from(group, false);
                    own_done = t < 0;
                }
                // from the back of the other ranges, nearest first: group + 1,
                // group - 1, group + 2, ...; none once every range is empty
                // (probing them all at the end of the walk cost ~0.1 ms)
                while (t < 0 && tried < ngroups - 1 &&
                       *(volatile unsigned *)empty < (unsigned)ngroups) {
                    const int d = tried / 2 + 1;
                    int v = (tried & 1) ? group - d : group + d;
                    v = ((v % ngroups) + ngroups) % ngroups;
                    t = take_from(v, true);
                    if (t < 0) ++tried;
                }
            }
            if (t < 0) t = nstatic + (int)atomicAdd(queue, 1u);
        }
        return __shfl_sync(FULL, t, 0);
    }
};

// One softened monopole term added to a particle slot's sums.
// SOFT: every system of the launch has eps > 0, so r2 >= eps^2 > 0 and the
// guard for a zero distance (eps = 0, coincident points) is not needed; the
// result is the same bit for bit.
template <bool KAHAN, bool POT, bool COUNT, bool SOFT = false>
__device__ __forceinline__ void interact(float m, float dx, float dy, float dz, float d2, float eps2,
                                         bool self, float &ax, float &ay, float &az, float &cx,
                                         float &cy, float &cz, float &pp, float &cp, unsigned &cnt)
{
    const float r2 = d2 + eps2;
    const float inv = SOFT ? rsqrtf(r2) : (r2 > 0.f ? rsqrtf(r2) : 0.f);
    const float mi = m * inv;
    const float mi3 = mi * inv * inv;
    acc_fma<KAHAN>(ax, cx, mi3, dx);
    acc_fma<KAHAN>(ay, cy, mi3, dy);
    acc_fma<KAHAN>(az, cz, mi3, dz);
    if (POT && !self) acc_add<KAHAN>(pp, cp, mi);
    if (COUNT) cnt += 1;
}

// A depth-cap bucket (equal keys down to level 21) is never taken as a whole:
// its particles are summed one by one, like the leaves they would be.
template <bool KAHAN, bool POT, bool COUNT, bool SOFT = false>
__device__ __forceinline__ void bucket_sum(const int4 *__restrict__ nodeR,
                                        const float4 *__restrict__ spos, int node, float px,
                                        float py, float pz, int myj, float eps2, float &ax,
                                        float &ay, float &az, float &cx, float &cy, float &cz,
                                        float &pp, float &cp, unsigned &cnt)
{
    const int4 R = __ldg(&nodeR[node]);  // first, count
    for (int q = R.x; q < R.x + R.y; ++q) {
        const float4 P = __ldg(&spos[q]);
        const float dx = P.x - px, dy = P.y - py, dz = P.z - pz;
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        interact<KAHAN, POT, COUNT, SOFT>(P.w, dx, dy, dz, d2, eps2, q == myj, ax, ay, az, cx,
                                          cy, cz, pp, cp, cnt);
    }
}

// Quadrupole mode: an accepted cell's monopole plus its second-order term.
// With d = com - x, s^2 = |d|^2 + eps^2 and I the cell's second moments about
// its centre of mass (FP32 copy: (xx, yy, zz, xy), (xz, yz, -, -)), the
// softened kernel expanded to second order gives, before the factor G,
//   a   += m d / s^3 - 3 (I d) / s^5 + ((15/2) (d.I.d) / s^7 - (3/2) tr I / s^5) d
//   phi -= m / s + (1/2) (3 (d.I.d) / s^5 - tr I / s^3)
// (the potential sum pp holds minus phi / G).
template <bool KAHAN, bool POT, bool COUNT>
__device__ __forceinline__ void interact_quad(const float4 *Qp, float m, float dx, float dy,
                                              float dz, float d2, float eps2, float &ax, float &ay,
                                              float &az, float &cx, float &cy, float &cz,
                                              float &pp, float &cp, unsigned &cnt)
{
    float q[8];
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(q[0]), "=f"(q[1]), "=f"(q[2]), "=f"(q[3]), "=f"(q[4]), "=f"(q[5]), "=f"(q[6]),
          "=f"(q[7])
        : "l"(Qp));
    const float r2 = d2 + eps2;
    const float inv = r2 > 0.f ? rsqrtf(r2) : 0.f;
    const float inv2 = inv * inv;
    const float inv3 = inv2 * inv;
    const float inv5 = inv3 * inv2;
    const float inv7 = inv5 * inv2;
    const float Id0 = fmaf(q[0], dx, fmaf(q[3], dy, q[4] * dz));
    const float Id1 = fmaf(q[3], dx, fmaf(q[1], dy, q[5] * dz));
    const float Id2 = fmaf(q[4], dx, fmaf(q[5], dy, q[2] * dz));
    const float dId = fmaf(dx, Id0, fmaf(dy, Id1, dz * Id2));
    const float tr = q[0] + q[1] + q[2];
    const float c = fmaf(7.5f * dId, inv7, fmaf(m, inv3, -1.5f * tr * inv5));
    const float t5 = -3.f * inv5;
    acc_add<KAHAN>(ax, cx, fmaf(c, dx, t5 * Id0));
    acc_add<KAHAN>(ay, cy, fmaf(c, dy, t5 * Id1));
    acc_add<KAHAN>(az, cz, fmaf(c, dz, t5 * Id2));
    if (POT) acc_add<KAHAN>(pp, cp, fmaf(m, inv, 0.5f * fmaf(3.f * dId, inv5, -tr * inv3)));
    if (COUNT) cnt += 1;
}

// GROUP = 32: the warp votes (__reduce_min_sync) on the next node and visits
// the union of its particles' traversals, one broadcast node load per step.
// GROUP = 4, 8, 16: aligned lane groups vote among themselves (xor-shuffle
// minimum) and each group walks the union of its own particles' traversals;
// a warp load then touches at most 32 / GROUP nodes.
// GROUP = 1: no vote; every lane advances through its own particles'
// traversal (loads diverge, no lane waits on nodes it does not need).
// Either way each particle visits exactly its own nodes in increasing index
// order, so its sums -- and the results -- do not depend on the shape.
// Register budget: a block of up to 512 threads, and enough blocks per SM
// for 48 resident warps with one particle per lane.
template <int PPL, int GROUP, bool KAHAN, bool POT, bool COUNT, bool OPEN = false,
          bool QUAD = false, bool SOFT = false>
__global__ void __launch_bounds__(512, PPL == 1 ? 3 : 2) k_walk(WalkArgs a)
{
    static_assert(GROUP == 1 || GROUP == 2 || GROUP == 4 || GROUP == 8 || GROUP == 16 ||
                      GROUP == 32,
                  "vote group: 1, 2, 4, 8, 16 or 32 lanes");
    // a lone particle per lane that walks alone is always the one at `cur`
    constexpr bool kSolo = PPL == 1 && GROUP == 1;
    const int lane = threadIdx.x & 31;
    Small *sm = a.small;
    if (sm->status) return;
    __shared__ unsigned s_next;
    if (threadIdx.x == 0) s_next = 0;
    __syncthreads();
    TileDealer deal(a, &s_next);
    for (;;) {
        const int t = deal.take(lane);
        if (t >= a.ntiles) break;
        const Tile tl = a.tiles[t];
        const SysStatic &S = a.sys[tl.sys];
        const int sstart = S.start;
        const int root = (int)a.noff[sstart];
        const int nend = (int)a.noff[sstart + S.n];
        const float eps2 = S.eps2;

        float px[PPL], py[PPL], pz[PPL];
        int nxt[PPL], myj[PPL];
        int leaf[PPL];  // OPEN: node index of the slot's own leaf (or bucket)
        float ax[PPL], ay[PPL], az[PPL], cx[PPL], cy[PPL], cz[PPL], pp[PPL], cp[PPL];
        unsigned cnt[PPL], vis[PPL];
        unsigned iters = 0;
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
            const int o = slot_offset<PPL, GROUP>(lane, k);
            myj[k] = tl.start + o;
            ax[k] = ay[k] = az[k] = cx[k] = cy[k] = cz[k] = pp[k] = cp[k] = 0.f;
            cnt[k] = vis[k] = 0;
            leaf[k] = -1;
            if (o < tl.count) {
                const float4 P = a.spos[myj[k]];
                px[k] = P.x; py[k] = P.y; pz[k] = P.z;
                nxt[k] = root;
                // the last node written at or before a particle is its leaf or
                // its bucket (particles inside a bucket start no nodes)
                if (OPEN) leaf[k] = (int)a.noff[myj[k] + 1] - 1;
            } else {
                px[k] = py[k] = pz[k] = 0.f;
                nxt[k] = nend;
            }
        }

        for (;;) {
            int cur = nxt[0];
#pragma unroll
            for (int k = 1; k < PPL; ++k) cur = min(cur, nxt[k]);
            if (GROUP == 32) {
                cur = (int)__reduce_min_sync(FULL, (unsigned)cur);
                if (cur >= nend) break;
            } else if (GROUP > 1) {
#pragma unroll
                for (int o = GROUP / 2; o > 0; o >>= 1) cur = min(cur, __shfl_xor_sync(FULL, cur, o));
                // every lane keeps executing the shuffles until the whole warp is done
                const bool done = cur >= nend;
                if (__all_sync(FULL, done)) break;
                if (done) continue;
            } else {
                if (cur >= nend) break;
            }
            if (COUNT) {
                ++iters;
#pragma unroll
                for (int k = 0; k < PPL; ++k) vis[k] += nxt[k] == cur;
            }
            float4 A;
            uint4 B;
            load_node(a.nodeW + cur, A, B);
            // skip > cur for every node (checked where the topology pass writes
            // it), so each step moves forward and the loop ends
            const int skip = wn_skip(B);
            const float crit = wn_crit(B);
            // low part of the centre of mass: int16 multiples of a power of two,
            // folded into the distance by one fused multiply-add per axis
            // (the product is exact, so this equals adding the decoded value)
            const float lscale = __int_as_float(B.w & 0x7f800000u);
            const float lqx = (float)(short)(B.z & 0xffffu);
            const float lqy = (float)(short)(B.z >> 16);
            const float lqz = (float)(short)(B.w & 0xffffu);
#pragma unroll
            for (int k = 0; k < PPL; ++k) {
                if (kSolo || nxt[k] == cur) {
                    // distance to the centre of mass from its high and low parts
                    const float dx = fmaf(lqx, lscale, A.x - px[k]);
                    const float dy = fmaf(lqy, lscale, A.y - py[k]);
                    const float dz = fmaf(lqz, lscale, A.z - pz[k]);
                    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    bool acc = fp32_accepts(d2, crit);
                    if (!acc && !fp32_opens(d2, crit))
                        acc = accept_fp64(a.nodeD, a.nodeR, a.nodeB, a.sys, a.dyn, tl.sys, cur,
                                          px[k], py[k], pz[k]);
                    // alternative rule: a cell holding the particle (its leaf lies in
                    // the cell's subtree, cur < leaf < skip) is always opened
                    if (OPEN && acc && crit >= 0.f && cur < leaf[k] && leaf[k] < skip) acc = false;
                    if (acc) {
                        // the potential leaves out the particle's own leaf
                        const bool self = POT && crit == kLeafCrit && __ldg(&a.nodeR[cur].x) == myj[k];
                        if (QUAD && crit >= 0.f)  // a cell, not a leaf
                            interact_quad<KAHAN, POT, COUNT>(a.nodeQ + 2 * (size_t)cur, A.w, dx, dy,
                                                             dz, d2, eps2, ax[k], ay[k], az[k],
                                                             cx[k], cy[k], cz[k], pp[k], cp[k],
                                                             cnt[k]);
                        else
                            interact<KAHAN, POT, COUNT, SOFT>(A.w, dx, dy, dz, d2, eps2, self,
                                                              ax[k], ay[k], az[k], cx[k], cy[k],
                                                              cz[k], pp[k], cp[k], cnt[k]);
                        nxt[k] = skip;
                    } else if (crit == kBucketCrit) {
                        bucket_sum<KAHAN, POT, COUNT, SOFT>(a.nodeR, a.spos, cur, px[k], py[k], pz[k],
                                                      myj[k], eps2, ax[k], ay[k], az[k], cx[k],
                                                      cy[k], cz[k], pp[k], cp[k], cnt[k]);
                        nxt[k] = skip;
                    } else {
                        nxt[k] = cur + 1;
                    }
                }
            }
        }

        if (COUNT) {
            unsigned long long ci = 0, cv = 0, it = iters;
#pragma unroll
            for (int k = 0; k < PPL; ++k) {
                const bool live = slot_offset<PPL, GROUP>(lane, k) < tl.count;
                ci += live ? cnt[k] : 0u;
                cv += live ? vis[k] : 0u;
            }
            for (int o = 16; o > 0; o >>= 1) {
                ci += __shfl_down_sync(FULL, ci, o);
                cv += __shfl_down_sync(FULL, cv, o);
                if (GROUP < 32) it = max(it, __shfl_down_sync(FULL, it, o));
            }
            if (lane == 0) {
                atomicAdd(&sm->wstats[0], ci);
                atomicAdd(&sm->wstats[1], it);
                atomicAdd(&sm->wstats[2], cv);
            }
        }
        const float G = S.G;
        float4 *acc = S.acc;
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
            const int o = slot_offset<PPL, GROUP>(lane, k);
            if (o < tl.count) {
                const uint32_t v = a.sid[myj[k]];
                if (COUNT) a.counts[v] = cnt[k];
                else acc[(int)v - sstart] = make_float4(G * ax[k], G * ay[k], G * az[k],
                                                        POT ? -G * pp[k] : 0.f);
            }
        }
    }
}

// ----------------------------------------------------- sibling-order walk
//
// One lane per particle, no vote, over the sibling-order copy of the records
// (a.nodeW; every node's children are neighbours, so lanes at sibling nodes
// share cache lines) and of the FP64 centres of mass (a.nodeD).  Each
// particle visits the same nodes in the same order as k_walk<1, 1> (first
// child on opening, the node after the subtree on acceptance), with the same
// arithmetic: a cell's threshold is formed from its level exactly as the
// topology pass forms the stored one, and a bucket reads its members through
// its depth-first index.  So results are bit-identical.  The loop ends
// because the build checked that the sibling order is a bijection of the
// depth-first order, whose walk ends (skip pointers increase).
// accept_fp64 for the sibling-order walk: the same FP64 test, with the cell's
// level and the system's side and theta^2 in hand and the centre of mass from
// the sibling-order copy.  (A call of its own keeps the other walks' register
// allocation around accept_fp64 as it was.)
__device__ __noinline__ bool accept_fp64_sib(const double4_32a *__restrict__ nodeD,
                                             const SysStatic *__restrict__ sys,
                                             const SysDyn *__restrict__ dyn, int sysid,
                                             unsigned cur, int level, float px, float py,
                                             float pz)
{
    const double theta2 = sys[sysid].theta2;
    const float side = dyn[sysid].side;
    const double4_32a D = nodeD[cur];
    const double dx = __dsub_rn(D.y, (double)px);
    const double dy = __dsub_rn(D.z, (double)py);
    const double dz = __dsub_rn(D.w, (double)pz);
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    const double s = (double)side * __longlong_as_double((long long)(1023 - level) << 52);
    return __dmul_rn(s, s) < __dmul_rn(theta2, d2);
}

template <bool KAHAN, bool POT, bool COUNT>
__global__ void __launch_bounds__(512, 3) k_walk_sib(WalkArgs a)
{
    const int lane = threadIdx.x & 31;
    Small *sm = a.small;
    if (sm->status) return;
    __shared__ unsigned s_next;
    if (threadIdx.x == 0) s_next = 0;
    __syncthreads();
    TileDealer deal(a, &s_next);
    for (;;) {
        const int t = deal.take(lane);
        if (t >= a.ntiles) break;
        const Tile tl = a.tiles[t];
        const SysStatic &S = a.sys[tl.sys];
        const int sstart = S.start;
        const float eps2 = S.eps2;
        const float inv_theta2 = S.inv_theta2;
        const float side = a.dyn[tl.sys].side;
        const int myj = tl.start + lane;
        const bool live = lane < tl.count;
        float px = 0.f, py = 0.f, pz = 0.f;
        unsigned cur = kSibEnd;
        if (live) {
            const float4 P = a.spos[myj];
            px = P.x; py = P.y; pz = P.z;
            cur = (unsigned)tl.sys;  // the system's root
        }
        float ax = 0.f, ay = 0.f, az = 0.f, cx = 0.f, cy = 0.f, cz = 0.f, pp = 0.f, cp = 0.f;
        unsigned cnt = 0, vis = 0, iters = 0;
        while (cur != kSibEnd) {
            if (COUNT) {
                ++iters;
                ++vis;
            }
            float4 A;
            uint4 B;
            load_node(a.nodeW + cur, A, B);
            const unsigned kind = (B.w >> 21) & 3u;
            const float lscale = __int_as_float(B.w & 0x7f800000u);
            const float lqx = (float)(short)(B.z & 0xffffu);
            const float lqy = (float)(short)(B.z >> 16);
            const float lqz = (float)(short)(B.w & 0xffffu);
            const float dx = fmaf(lqx, lscale, A.x - px);
            const float dy = fmaf(lqy, lscale, A.y - py);
            const float dz = fmaf(lqz, lscale, A.z - pz);
            const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            // the threshold k_walk reads from the record: a cell's from its
            // level (the topology pass's formula), -1 for a leaf, +inf for a
            // bucket; the same branch structure follows, so leaves and
            // accepted cells share one interaction path
            const int level = (int)((B.w >> 16) & 31u);
            const float sl = __fmul_rn(side, __int_as_float((127 - level) << 23));
            const float ccell = __fmul_rn(__fmul_rn(sl, sl), inv_theta2);
            const float crit = kind == kSibCell ? ccell : (kind == kSibLeaf ? kLeafCrit : kBucketCrit);
            bool acc = fp32_accepts(d2, crit);
            if (!acc && !fp32_opens(d2, crit))
                acc = accept_fp64_sib(a.nodeD, a.sys, a.dyn, tl.sys, cur, level, px, py, pz);
            if (acc) {
                const bool self = POT && kind == kSibLeaf && (int)B.x == myj;
                interact<KAHAN, POT, COUNT>(A.w, dx, dy, dz, d2, eps2, self, ax, ay, az, cx, cy, cz,
                                            pp, cp, cnt);
                cur = B.y;
            } else if (kind == kSibBucket) {
                bucket_sum<KAHAN, POT, COUNT>(a.nodeR, a.spos, (int)B.x, px, py, pz, myj, eps2,
                                              ax, ay, az, cx, cy, cz, pp, cp, cnt);
                cur = B.y;
            } else {
                cur = B.x;
            }
        }
        if (COUNT) {
            unsigned long long ci = live ? cnt : 0u, cv = live ? vis : 0u, it = iters;
            for (int o = 16; o > 0; o >>= 1) {
                ci += __shfl_down_sync(FULL, ci, o);
                cv += __shfl_down_sync(FULL, cv, o);
                it = max(it, __shfl_down_sync(FULL, it, o));
            }
            if (lane == 0) {
                atomicAdd(&sm->wstats[0], ci);
                atomicAdd(&sm->wstats[1], it);
                atomicAdd(&sm->wstats[2], cv);
            }
        }
        if (live) {
            const uint32_t v = a.sid[myj];
            const float G = S.G;
            if (COUNT) a.counts[v] = cnt;
            else S.acc[(int)v - sstart] = make_float4(G * ax, G * ay, G * az,
                                                      POT ? -G * pp : 0.f);
        }
    }
}

// ---------------------------------------------------------------- split walk
//
// The same per-particle decisions and the same interaction set as k_walk, in
// two phases per tile of 32 particles:
//   1. the top levels (<= Ltop): the warp votes on the smallest next node
//      (__reduce_min_sync) and reads it once for all lanes; every lane decides
//      for itself.  A lane that opens a level-Ltop node does not descend: the
//      warp appends (first child, subtree end) to its queue in shared memory,
//      and every lane that opened it sets the entry's bit in its own mask.
//   2. the levels below: every lane walks the queued subtrees its bit is set
//      in, one after another, on its own (no vote, no waiting on other lanes).
// The top levels are where the walks of neighbouring particles coincide
// (a broadcast load serves the whole warp); below, they diverge, and the lanes
// stop sharing a schedule.  A full queue is drained (phase 2) before phase 1
// goes on.  A particle's terms are summed (Kahan) in an order fixed by its
// tile -- 32 consecutive particles of its system, whatever the launch shape,
// alone or in a forest -- so results are bit-identical across split shapes.
constexpr int kSplitQueue = 32;       // queue entries per warp
constexpr int kSplitMaxWarps = 16;    // warps per block

// Lowest level walked by the warp vote: 3 levels above the depth at which a
// uniform system has about one particle per cell (floor(log8 n)), within 2..5.
__device__ __forceinline__ int split_top_level(int n)
{
    const int l8 = (31 - __clz(max(n, 1))) / 3;
    return min(5, max(2, l8 - 3));
}

template <bool KAHAN, bool POT, bool COUNT, bool SOFT = false>
__global__ void __launch_bounds__(512, 3) k_walk_split(WalkArgs a)
{
    __shared__ uint2 s_q[kSplitMaxWarps][kSplitQueue];  // (first child, subtree end)
    __shared__ unsigned s_next;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    Small *sm = a.small;
    if (sm->status) return;
    if (threadIdx.x == 0) s_next = 0;
    __syncthreads();
    TileDealer deal(a, &s_next);
    for (;;) {
        const int t = deal.take(lane);
        if (t >= a.ntiles) break;
        const Tile tl = a.tiles[t];
        const int sysid = tl.sys;
        int root, nend;
        float eps2, crit_top;
        {
            const SysStatic &S = a.sys[sysid];
            root = (int)a.noff[S.start];
            nend = (int)a.noff[S.start + S.n];
            eps2 = S.eps2;
            // threshold of the level-Ltop nodes, by the topology pass's formula
            const float sl = __fmul_rn(a.dyn[sysid].side,
                                       __int_as_float((127 - split_top_level(S.n)) << 23));
            crit_top = __fmul_rn(__fmul_rn(sl, sl), S.inv_theta2);
        }

        const int myj = tl.start + lane;
        const bool live = lane < tl.count;
        float px = 0.f, py = 0.f, pz = 0.f;
        if (live) {
            const float4 P = a.spos[myj];
            px = P.x; py = P.y; pz = P.z;
        }
        float ax = 0.f, ay = 0.f, az = 0.f, cx = 0.f, cy = 0.f, cz = 0.f, pp = 0.f, cp = 0.f;
        unsigned cnt = 0, iters = 0, vis = 0;
        int nxt = live ? root : nend;
        int qn = 0;           // warp-uniform
        unsigned mybits = 0;  // bit k: this lane opened the node of queue entry k
        bool top_done = false;

        for (;;) {
            // ---- phase 1: warp-voted walk of the top levels
            while (qn < kSplitQueue) {
                const int cur = (int)__reduce_min_sync(FULL, (unsigned)nxt);
                if (cur >= nend) {
                    top_done = true;
                    break;
                }
                if (COUNT) ++iters;
                float4 A;
                uint4 B;
                load_node(a.nodeW + cur, A, B);
                const int skip = wn_skip(B);  // > cur, checked by the topology pass
                const float crit = wn_crit(B);
                bool enq = false;
                if (nxt == cur) {
                    if (COUNT) ++vis;
                    const float lscale = __int_as_float(B.w & 0x7f800000u);
                    const float dx = fmaf((float)(short)(B.z & 0xffffu), lscale, A.x - px);
                    const float dy = fmaf((float)(short)(B.z >> 16), lscale, A.y - py);
                    const float dz = fmaf((float)(short)(B.w & 0xffffu), lscale, A.z - pz);
                    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    bool acc = fp32_accepts(d2, crit);
                    if (!acc && !fp32_opens(d2, crit))
                        acc = accept_fp64(a.nodeD, a.nodeR, a.nodeB, a.sys, a.dyn, sysid, cur,
                                          px, py, pz);
                    if (acc) {
                        const bool self = POT && crit == kLeafCrit && __ldg(&a.nodeR[cur].x) == myj;
                        interact<KAHAN, POT, COUNT, SOFT>(A.w, dx, dy, dz, d2, eps2, self, ax, ay, az,
                                                    cx, cy, cz, pp, cp, cnt);
                        nxt = skip;
                    } else if (crit == crit_top) {
                        enq = true;
                        nxt = skip;
                    } else if (crit == kBucketCrit) {
                        bucket_sum<KAHAN, POT, COUNT, SOFT>(a.nodeR, a.spos, cur, px, py, pz, myj, eps2,
                                                      ax, ay, az, cx, cy, cz, pp, cp, cnt);
                        nxt = skip;
                    } else {
                        nxt = cur + 1;
                    }
                }
                if (__any_sync(FULL, enq)) {
                    if (lane == 0) s_q[warp][qn] = make_uint2((unsigned)cur + 1u, (unsigned)skip);
                    mybits |= (enq ? 1u : 0u) << qn;
                    ++qn;
                }
            }
            __syncwarp();
            if (qn > 0) {
                // ---- phase 2: every lane walks its queued subtrees
                int n2 = 0, e2 = 0;
                unsigned it2 = 0;
                for (;;) {
                    if (n2 >= e2) {  // next queued subtree of this lane (never empty)
                        if (!mybits) break;
                        const uint2 E = s_q[warp][__ffs(mybits) - 1];
                        mybits &= mybits - 1u;
                        n2 = (int)E.x;
                        e2 = (int)E.y;
                    }
                    if (COUNT) {
                        ++it2;
                        ++vis;
                    }
                    float4 A;
                    uint4 B;
                    load_node(a.nodeW + n2, A, B);
                    const int skip = wn_skip(B);  // > n2, checked by the topology pass
                    const float crit = wn_crit(B);
                    const float lscale = __int_as_float(B.w & 0x7f800000u);
                    const float dx = fmaf((float)(short)(B.z & 0xffffu), lscale, A.x - px);
                    const float dy = fmaf((float)(short)(B.z >> 16), lscale, A.y - py);
                    const float dz = fmaf((float)(short)(B.w & 0xffffu), lscale, A.z - pz);
                    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    bool acc = fp32_accepts(d2, crit);
                    if (!acc && !fp32_opens(d2, crit))
                        acc = accept_fp64(a.nodeD, a.nodeR, a.nodeB, a.sys, a.dyn, sysid, n2,
                                          px, py, pz);
                    if (acc) {
                        const bool self = POT && crit == kLeafCrit && __ldg(&a.nodeR[n2].x) == myj;
                        interact<KAHAN, POT, COUNT, SOFT>(A.w, dx, dy, dz, d2, eps2, self, ax, ay, az,
                                                    cx, cy, cz, pp, cp, cnt);
                        n2 = skip;
                    } else if (crit == kBucketCrit) {
                        bucket_sum<KAHAN, POT, COUNT, SOFT>(a.nodeR, a.spos, n2, px, py, pz, myj, eps2,
                                                      ax, ay, az, cx, cy, cz, pp, cp, cnt);
                        n2 = skip;
                    } else {
                        n2 = n2 + 1;
                    }
                }
                if (COUNT) {
                    // warp iterations of the phase: the slowest lane's
                    for (int o = 16; o > 0; o >>= 1) it2 = max(it2, __shfl_xor_sync(FULL, it2, o));
                    iters += it2;
                }
                qn = 0;
                mybits = 0;
                __syncwarp();
            }
            if (top_done) break;
        }

        if (COUNT) {
            unsigned long long ci = live ? cnt : 0u, cv = live ? vis : 0u;
            for (int o = 16; o > 0; o >>= 1) {
                ci += __shfl_down_sync(FULL, ci, o);
                cv += __shfl_down_sync(FULL, cv, o);
            }
            if (lane == 0) {
                atomicAdd(&sm->wstats[0], ci);
                atomicAdd(&sm->wstats[1], (unsigned long long)iters);
                atomicAdd(&sm->wstats[2], cv);
            }
        }
        if (live) {
            const uint32_t v = a.sid[myj];
            const SysStatic &S = a.sys[sysid];
            const float G = S.G;
            if (COUNT) a.counts[v] = cnt;
            else S.acc[(int)v - S.start] = make_float4(G * ax, G * ay, G * az, POT ? -G * pp : 0.f);
        }
        __syncwarp();
    }
}

// ------------------------------------------------------ interaction lists
//
// The paper's two-phase form (a flattened tree walked into interaction
// lists, then the lists evaluated), per tile of 32 particles and exact per
// particle:
//   1. the warp walks the union of its particles' traversals (vote on the
//      smallest next index, one broadcast node load per step, every lane
//      decides for itself) and appends each node that some lane takes --
//      accepted cell, leaf or depth-cap bucket -- with the mask of the lanes
//      that take it, to a list in shared memory;
//   2. the warp evaluates the list in order: one broadcast load per entry,
//      and every lane whose bit is set adds the term, with no decisions left.
// A full list is evaluated before the walk goes on.  Every particle adds its
// own terms in depth-first order, as in k_walk, so results are bit-identical
// to every other shape with a vote group.
constexpr int kListCap = 128;      // entries per warp
constexpr int kListMaxWarps = 16;  // warps per block

template <bool KAHAN, bool POT, bool COUNT>
__global__ void __launch_bounds__(512, 3) k_walk_list(WalkArgs a)
{
    __shared__ uint2 s_list[kListMaxWarps][kListCap];  // (node, lane mask)
    __shared__ unsigned s_next;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    Small *sm = a.small;
    if (sm->status) return;
    if (threadIdx.x == 0) s_next = 0;
    __syncthreads();
    TileDealer deal(a, &s_next);
    for (;;) {
        const int t = deal.take(lane);
        if (t >= a.ntiles) break;
        const Tile tl = a.tiles[t];
        const int sysid = tl.sys;
        int root, nend;
        float eps2;
        {
            const SysStatic &S = a.sys[sysid];
            root = (int)a.noff[S.start];
            nend = (int)a.noff[S.start + S.n];
            eps2 = S.eps2;
        }
        const int myj = tl.start + lane;
        const bool live = lane < tl.count;
        float px = 0.f, py = 0.f, pz = 0.f;
        if (live) {
            const float4 P = a.spos[myj];
            px = P.x; py = P.y; pz = P.z;
        }
        float ax = 0.f, ay = 0.f, az = 0.f, cx = 0.f, cy = 0.f, cz = 0.f, pp = 0.f, cp = 0.f;
        unsigned cnt = 0, iters = 0, vis = 0;
        int nxt = live ? root : nend;
        bool done = false;
        while (!done) {
            // ---- phase 1: walk the union, list what the lanes take
            int n = 0;  // warp-uniform
            while (n < kListCap) {
                const int cur = (int)__reduce_min_sync(FULL, (unsigned)nxt);
                if (cur >= nend) {
                    done = true;
                    break;
                }
                if (COUNT) ++iters;
                float4 A;
                uint4 B;
                load_node(a.nodeW + cur, A, B);
                const int skip = wn_skip(B);  // > cur, checked by the topology pass
                const float crit = wn_crit(B);
                bool take = false;
                if (nxt == cur) {
                    if (COUNT) ++vis;
                    const float lscale = __int_as_float(B.w & 0x7f800000u);
                    const float dx = fmaf((float)(short)(B.z & 0xffffu), lscale, A.x - px);
                    const float dy = fmaf((float)(short)(B.z >> 16), lscale, A.y - py);
                    const float dz = fmaf((float)(short)(B.w & 0xffffu), lscale, A.z - pz);
                    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    bool acc = fp32_accepts(d2, crit);
                    if (!acc && !fp32_opens(d2, crit))
                        acc = accept_fp64(a.nodeD, a.nodeR, a.nodeB, a.sys, a.dyn, sysid, cur,
                                          px, py, pz);
                    take = acc || crit == kBucketCrit;
                    nxt = take ? skip : cur + 1;
                }
                const unsigned m = __ballot_sync(FULL, take);
                if (m) {
                    if (lane == 0) s_list[warp][n] = make_uint2((unsigned)cur, m);
                    ++n;
                }
            }
            __syncwarp();
            // ---- phase 2: evaluate the list, entry by entry in walk order
            for (int e = 0; e < n; ++e) {
                const uint2 E = s_list[warp][e];
                if (COUNT) ++iters;
                float4 A;
                uint4 B;
                load_node(a.nodeW + E.x, A, B);
                if (!((E.y >> lane) & 1u)) continue;
                const float crit = wn_crit(B);
                if (crit == kBucketCrit) {
                    bucket_sum<KAHAN, POT, COUNT>(a.nodeR, a.spos, (int)E.x, px, py, pz, myj, eps2,
                                                  ax, ay, az, cx, cy, cz, pp, cp, cnt);
                    continue;
                }
                const float lscale = __int_as_float(B.w & 0x7f800000u);
                const float dx = fmaf((float)(short)(B.z & 0xffffu), lscale, A.x - px);
                const float dy = fmaf((float)(short)(B.z >> 16), lscale, A.y - py);
                const float dz = fmaf((float)(short)(B.w & 0xffffu), lscale, A.z - pz);
                const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                const bool self = POT && crit == kLeafCrit && __ldg(&a.nodeR[E.x].x) == myj;
                interact<KAHAN, POT, COUNT>(A.w, dx, dy, dz, d2, eps2, self, ax, ay, az, cx, cy,
                                            cz, pp, cp, cnt);
            }
            __syncwarp();
        }

        if (COUNT) {
            unsigned long long ci = live ? cnt : 0u, cv = live ? vis : 0u;
            for (int o = 16; o > 0; o >>= 1) {
                ci += __shfl_down_sync(FULL, ci, o);
                cv += __shfl_down_sync(FULL, cv, o);
            }
            if (lane == 0) {
                atomicAdd(&sm->wstats[0], ci);
                atomicAdd(&sm->wstats[1], (unsigned long long)iters);
                atomicAdd(&sm->wstats[2], cv);
            }
        }
        if (live) {
            const uint32_t v = a.sid[myj];
            const SysStatic &S = a.sys[sysid];
            const float G = S.G;
            if (COUNT) a.counts[v] = cnt;
            else S.acc[(int)v - S.start] = make_float4(G * ax, G * ay, G * az, POT ? -G * pp : 0.f);
        }
        __syncwarp();
    }
}

// A cached occupancy: computed once per (variant, block size), -1 when the
// shape does not fit.  Host threads may race here (the server's thread and
// the caller's); at worst both compute the same value.
template <class F>
int cached_occupancy(std::atomic<int> &slot, F compute)
{
    int c = slot.load(std::memory_order_relaxed);
    if (c == 0) {
        const int occ = compute();
        c = occ > 0 ? occ : -1;
        slot.store(c, std::memory_order_relaxed);
    }
    return c > 0 ? c : 0;
}

constexpr int kMaxWalkWarps = 48;

// Blocks of `warps` warps that fit on one SM, queried once per variant and
// block size (never during stream capture: callers query before capturing).
template <int PPL, int GROUP, bool KAHAN, bool POT, bool COUNT, bool OPEN = false,
          bool QUAD = false, bool SOFT = false>
int occupancy(int warps)
{
    static std::atomic<int> cache[33];
    if (warps < 1 || warps > 32) return 0;
    return cached_occupancy(cache[warps], [warps] {
        auto *fn = k_walk<PPL, GROUP, KAHAN, POT, COUNT, OPEN, QUAD, SOFT>;
        // the walk uses no shared memory: give the SM's unified storage to L1
        cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, warps * 32, 0) != cudaSuccess)
            occ = 0;
        // at most 48 resident warps: the walk is bound by L1's throughput
        // for scattered node loads, and 64 warps (where registers allow
        // them) lower the L1 hit rate more than they hide latency
        // (uniform cube of 2^20, theta 0.5: 2.79 ms at 64 warps, 2.70 at 48)
        return occ * warps > kMaxWalkWarps ? std::max(1, kMaxWalkWarps / warps) : occ;
    });
}

// The split walk needs its queue and parked sums in shared memory: ask for
// the smallest carveout that still holds the blocks the registers allow.
template <bool KAHAN, bool POT, bool COUNT, bool SOFT = false>
int occupancy_split(int warps)
{
    static std::atomic<int> cache[33];
    if (warps < 1 || warps > kSplitMaxWarps) return 0;
    return cached_occupancy(cache[warps], [warps] {
        auto *fn = k_walk_split<KAHAN, POT, COUNT, SOFT>;
        cudaFuncAttributes fa{};
        int occ = 0;
        if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess) {
            const int regs = fa.numRegs > 0 ? fa.numRegs : 64;
            const int per_sm = 65536 / (regs * warps * 32);
            const int want = per_sm < 1 ? 1 : (per_sm > 64 / warps ? 64 / warps : per_sm);
            const size_t need = (size_t)want * (fa.sharedSizeBytes + 1024) * 100;
            const int pct = (int)((need + 228 * 1024 - 1) / (228 * 1024));
            cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 pct > 100 ? 100 : pct);
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, warps * 32, 0) != cudaSuccess)
                occ = 0;
        }
        return occ;
    });
}

template <bool KAHAN, bool POT, bool COUNT, bool SOFT = false>
int launch_split(const WalkArgs *a, const WalkShape &sh, int nsm, cudaStream_t st)
{
    if (sh.ppl != 1) return 0;
    const int occ = occupancy_split<KAHAN, POT, COUNT, SOFT>(sh.warps);
    if (occ <= 0) return 0;
    if (a) {
        const int bps = sh.blocks_per_sm > 0 ? sh.blocks_per_sm : occ;
        k_walk_split<KAHAN, POT, COUNT, SOFT><<<nsm * bps, sh.warps * 32, 0, st>>>(*a);
    }
    return occ;
}

template <bool KAHAN, bool POT, bool COUNT>
int occupancy_sib(int warps)
{
    static std::atomic<int> cache[33];
    if (warps < 1 || warps > 16) return 0;
    return cached_occupancy(cache[warps], [warps] {
        auto *fn = k_walk_sib<KAHAN, POT, COUNT>;
        cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, warps * 32, 0) != cudaSuccess)
            occ = 0;
        return occ;
    });
}

template <bool KAHAN, bool POT, bool COUNT>
int launch_sib(const WalkArgs *a, const WalkShape &sh, int nsm, cudaStream_t st)
{
    if (sh.ppl != 1) return 0;
    const int occ = occupancy_sib<KAHAN, POT, COUNT>(sh.warps);
    if (occ <= 0) return 0;
    if (a) {
        const int bps = sh.blocks_per_sm > 0 ? sh.blocks_per_sm : occ;
        k_walk_sib<KAHAN, POT, COUNT><<<nsm * bps, sh.warps * 32, 0, st>>>(*a);
    }
    return occ;
}

template <bool KAHAN, bool POT, bool COUNT>
int occupancy_list(int warps)
{
    static std::atomic<int> cache[33];
    if (warps < 1 || warps > kListMaxWarps) return 0;
    return cached_occupancy(cache[warps], [warps] {
        auto *fn = k_walk_list<KAHAN, POT, COUNT>;
        cudaFuncAttributes fa{};
        int occ = 0;
        if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess) {
            const int regs = fa.numRegs > 0 ? fa.numRegs : 64;
            const int per_sm = 65536 / (regs * warps * 32);
            const int want = per_sm < 1 ? 1 : (per_sm > 64 / warps ? 64 / warps : per_sm);
            const size_t need = (size_t)want * (fa.sharedSizeBytes + 1024) * 100;
            const int pct = (int)((need + 228 * 1024 - 1) / (228 * 1024));
            cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 pct > 100 ? 100 : pct);
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, warps * 32, 0) != cudaSuccess)
                occ = 0;
        }
        return occ;
    });
}

template <bool KAHAN, bool POT, bool COUNT>
int launch_list(const WalkArgs *a, const WalkShape &sh, int nsm, cudaStream_t st)
{
    if (sh.ppl != 1) return 0;
    const int occ = occupancy_list<KAHAN, POT, COUNT>(sh.warps);
    if (occ <= 0) return 0;
    if (a) {
        const int bps = sh.blocks_per_sm > 0 ? sh.blocks_per_sm : occ;
        k_walk_list<KAHAN, POT, COUNT><<<nsm * bps, sh.warps * 32, 0, st>>>(*a);
    }
    return occ;
}

template <int PPL, int GROUP, bool KAHAN, bool POT, bool COUNT, bool OPEN = false,
          bool QUAD = false, bool SOFT = false>
void launch_one(const WalkArgs &a, const WalkShape &sh, int nsm, cudaStream_t st)
{
    const int threads = sh.warps * 32;
    int bps = sh.blocks_per_sm;
    if (bps <= 0) bps = occupancy<PPL, GROUP, KAHAN, POT, COUNT, OPEN, QUAD, SOFT>(sh.warps);
    if (bps <= 0) bps = 1;
    k_walk<PPL, GROUP, KAHAN, POT, COUNT, OPEN, QUAD, SOFT><<<nsm * bps, threads, 0, st>>>(a);
}

template <bool KAHAN, bool POT, bool COUNT, bool OPEN, bool QUAD>
int fixed_one(const WalkArgs *a, const WalkShape &sh, int nsm, cudaStream_t st)
{
    if (a) launch_one<1, 1, KAHAN, POT, COUNT, OPEN, QUAD>(*a, sh, nsm, st);
    return occupancy<1, 1, KAHAN, POT, COUNT, OPEN, QUAD>(sh.warps);
}

// The walks with a fixed shape (one particle per lane, no vote): the
// alternative opening rule (BH_OPEN_INSIDE) and the quadrupole term
// (BH_QUADRUPOLE, Kahan sums only).  Counting needs no quadrupole term: the
// accepted sets are the same.
template <bool COUNT>
int run_fixed(bool kahan, bool pot, const WalkArgs *a, const WalkShape &sh, int nsm,
              cudaStream_t st)
{
    if (sh.ppl != 1 || sh.group != 1) return 0;
    const bool open = sh.open_inside;
    if (COUNT)
        return open ? fixed_one<true, false, true, true, false>(a, sh, nsm, st)
                    : fixed_one<true, false, true, false, false>(a, sh, nsm, st);
    if (sh.quad) {
        if (!kahan) return 0;
        if (open)
            return pot ? fixed_one<true, true, false, true, true>(a, sh, nsm, st)
                       : fixed_one<true, false, false, true, true>(a, sh, nsm, st);
        return pot ? fixed_one<true, true, false, false, true>(a, sh, nsm, st)
                   : fixed_one<true, false, false, false, true>(a, sh, nsm, st);
    }
    if (kahan && pot) return fixed_one<true, true, false, true, false>(a, sh, nsm, st);
    if (kahan) return fixed_one<true, false, false, true, false>(a, sh, nsm, st);
    if (pot) return fixed_one<false, true, false, true, false>(a, sh, nsm, st);
    return fixed_one<false, false, false, true, false>(a, sh, nsm, st);
}

// Dispatch of the runtime shape onto the compiled variants.
template <bool COUNT>
struct Variants {
    template <int PPL, int GROUP>
    static int pick(bool kahan, bool pot, const WalkArgs *a, const WalkShape &sh, int nsm,
                    cudaStream_t st)
    {
        if (COUNT) {
            if (a) launch_one<PPL, GROUP, true, false, true>(*a, sh, nsm, st);
            return occupancy<PPL, GROUP, true, false, true>(sh.warps);
        }
        // one particle per lane without a vote and eps > 0 everywhere: the
        // variant without the zero-distance guard (the same results)
        if (PPL == 1 && GROUP == 1 && sh.soft && kahan) {
            if (pot) {
                if (a) launch_one<1, 1, true, true, false, false, false, true>(*a, sh, nsm, st);
                return occupancy<1, 1, true, true, false, false, false, true>(sh.warps);
            }
            if (a) launch_one<1, 1, true, false, false, false, false, true>(*a, sh, nsm, st);
            return occupancy<1, 1, true, false, false, false, false, true>(sh.warps);
        }
        if (kahan && pot) {
            if (a) launch_one<PPL, GROUP, true, true, false>(*a, sh, nsm, st);
            return occupancy<PPL, GROUP, true, true, false>(sh.warps);
        }
        if (kahan) {
            if (a) launch_one<PPL, GROUP, true, false, false>(*a, sh, nsm, st);
            return occupancy<PPL, GROUP, true, false, false>(sh.warps);
        }
        if (pot) {
            if (a) launch_one<PPL, GROUP, false, true, false>(*a, sh, nsm, st);
            return occupancy<PPL, GROUP, false, true, false>(sh.warps);
        }
        if (a) launch_one<PPL, GROUP, false, false, false>(*a, sh, nsm, st);
        return occupancy<PPL, GROUP, false, false, false>(sh.warps);
    }

    // returns the occupancy of the variant (0 = shape not supported)
    static int run(bool kahan, bool pot, const WalkArgs *a, const WalkShape &sh, int nsm,
                   cudaStream_t st)
    {
        if (sh.open_inside || sh.quad) return run_fixed<COUNT>(kahan, pot, a, sh, nsm, st);
        if (sh.group == BH_GROUP_LIST) {  // interaction lists
            if (COUNT) return launch_list<true, false, true>(a, sh, nsm, st);
            if (kahan && pot) return launch_list<true, true, false>(a, sh, nsm, st);
            if (kahan) return launch_list<true, false, false>(a, sh, nsm, st);
            if (pot) return launch_list<false, true, false>(a, sh, nsm, st);
            return launch_list<false, false, false>(a, sh, nsm, st);
        }
        if (sh.group == BH_GROUP_SIBLINGS) {  // one lane per particle, sibling-order records
            if (COUNT) return launch_sib<true, false, true>(a, sh, nsm, st);
            if (kahan && pot) return launch_sib<true, true, false>(a, sh, nsm, st);
            if (kahan) return launch_sib<true, false, false>(a, sh, nsm, st);
            if (pot) return launch_sib<false, true, false>(a, sh, nsm, st);
            return launch_sib<false, false, false>(a, sh, nsm, st);
        }
        if (sh.group == 0) {  // split walk
            if (COUNT) return launch_split<true, false, true>(a, sh, nsm, st);
            if (kahan && pot) return launch_split<true, true, false>(a, sh, nsm, st);
            // eps > 0 everywhere: the variant without the zero-distance guard
            if (kahan && sh.soft) return launch_split<true, false, false, true>(a, sh, nsm, st);
            if (kahan) return launch_split<true, false, false>(a, sh, nsm, st);
            if (pot) return launch_split<false, true, false>(a, sh, nsm, st);
            return launch_split<false, false, false>(a, sh, nsm, st);
        }
        if (COUNT) {
            if (sh.ppl != 1) return 0;
            switch (sh.group) {
                case 1: return pick<1, 1>(kahan, pot, a, sh, nsm, st);
                case 2: return pick<1, 2>(kahan, pot, a, sh, nsm, st);
                case 4: return pick<1, 4>(kahan, pot, a, sh, nsm, st);
                case 8: return pick<1, 8>(kahan, pot, a, sh, nsm, st);
                case 32: return pick<1, 32>(kahan, pot, a, sh, nsm, st);
            }
            return 0;
        }
        const int key = sh.group * 8 + sh.ppl;
        switch (key) {
            case 1 * 8 + 1: return pick<1, 1>(kahan, pot, a, sh, nsm, st);
            case 1 * 8 + 2: return pick<2, 1>(kahan, pot, a, sh, nsm, st);
            case 1 * 8 + 4: return pick<4, 1>(kahan, pot, a, sh, nsm, st);
            case 2 * 8 + 1: return pick<1, 2>(kahan, pot, a, sh, nsm, st);
            case 4 * 8 + 1: return pick<1, 4>(kahan, pot, a, sh, nsm, st);
            case 4 * 8 + 2: return pick<2, 4>(kahan, pot, a, sh, nsm, st);
            case 8 * 8 + 1: return pick<1, 8>(kahan, pot, a, sh, nsm, st);
            case 8 * 8 + 2: return pick<2, 8>(kahan, pot, a, sh, nsm, st);
            case 32 * 8 + 1: return pick<1, 32>(kahan, pot, a, sh, nsm, st);
            case 32 * 8 + 2: return pick<2, 32>(kahan, pot, a, sh, nsm, st);
            case 32 * 8 + 4: return pick<4, 32>(kahan, pot, a, sh, nsm, st);
        }
        return 0;
    }
};

}  // namespace

int launch_walk(const WalkArgs &a, const WalkShape &sh, bool kahan, bool pot, bool count,
                int nsm, cudaStream_t st)
{
    const int occ = count ? Variants<true>::run(kahan, pot, &a, sh, nsm, st)
                          : Variants<false>::run(kahan, pot, &a, sh, nsm, st);
    if (occ <= 0) return -1;
    g_launches += 1;
    return 1;
}

int walk_max_blocks_per_sm(const WalkShape &sh, bool kahan, bool pot)
{
    WalkShape cs = sh;
    cs.ppl = 1;
    if (cs.open_inside || cs.quad) cs.group = 1;
    Variants<true>::run(true, false, nullptr, cs, 0, nullptr);  // the counting variant too
    return Variants<false>::run(kahan, pot, nullptr, sh, 0, nullptr);
}

}  // namespace bh
