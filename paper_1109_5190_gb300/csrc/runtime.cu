// runtime.cu -- host runtime behind the C ABI of include/bh.h.
//
// One internal object, Forest, runs every path: a single system is a forest
// of one; a bh_forest is many systems sharing every launch of a step; the
// server re-tables its resident systems into a forest at every tick.  A step
// enqueues, on the forest's own stream:
//   kick+drift fused with the box / root reductions -> per-system cube ->
//   Morton keys -> 8-pass segmented radix sort -> gather into Morton order ->
//   topology (count, scan, capacity check, write) -> centre of mass, one
//   launch per level -> persistent walk -> closing kick.
// Node buffers have a capacity; a step whose tree would not fit sets a device
// status, every later kernel of the run returns at once, and the host rolls
// the failed step back (positions and velocities saved at its start), grows
// the buffers and redoes the remaining steps.  Graph mode captures the step
// loop once per (step count, buffers, launch shape) and replays it.
#include "bh.h"
#include "bh_internal.cuh"

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <condition_variable>
#include <cstddef>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

using namespace bh;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

#define CKR(call)                                                                        \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            cudaGetLastError();                                                          \
            return fail(BH_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
        }                                                                                \
    } while (0)

#define TRY(expr)                 \
    do {                          \
        int rc_ = (expr);         \
        if (rc_ != BH_OK) return rc_; \
    } while (0)

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    int ensure(size_t nb)
    {
        if (nb == 0) nb = 256;
        if (p && nb <= bytes) return BH_OK;
        release();
        cudaError_t e = cudaMalloc(&p, nb);
        if (e != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            return fail(BH_ERR_OOM, "cudaMalloc of " + std::to_string(nb) + " bytes failed: " +
                                        cudaGetErrorString(e));
        }
        bytes = nb;
        return BH_OK;
    }
    template <class T>
    T *as() const { return static_cast<T *>(p); }
};

bool finite_state(int64_t n, const float *pm, const float *vel)
{
    for (int64_t i = 0; i < n; ++i) {
        const float *p = pm + 4 * i;
        if (!(std::isfinite(p[0]) && std::isfinite(p[1]) && std::isfinite(p[2]) &&
              std::isfinite(p[3]) && p[3] > 0.f))
            return false;
        if (vel) {
            const float *v = vel + 4 * i;
            if (!(std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]))) return false;
        }
    }
    return true;
}

int check_params(double G, double eps, double theta)
{
    if (!(G > 0.0) || !std::isfinite(G)) return fail(BH_ERR_INVALID, "G must be finite and > 0");
    if (!(eps >= 0.0) || !std::isfinite(eps)) return fail(BH_ERR_INVALID, "eps must be finite and >= 0");
    if (!(theta >= 0.0) || !std::isfinite(theta))
        return fail(BH_ERR_INVALID, "theta must be finite and >= 0");
    return BH_OK;
}

// Particle state of one system: pos, vel, acc, backup pos, backup vel.  The
// five arrays live in memory the state owns (alloc) or in a region of a pool
// that outlives it (place: the server's pool carved from its HBM budget).
struct SysState {
    int64_t n = 0;
    DevBuf mem;
    float4 *ext = nullptr;
    double G = 1.0, eps = 0.01, theta = 0.5, dt = 1e-3;
    float4 *pos() const { return ext ? ext : mem.as<float4>(); }
    float4 *vel() const { return pos() + n; }
    float4 *acc() const { return pos() + 2 * n; }
    float4 *bpos() const { return pos() + 3 * n; }
    float4 *bvel() const { return pos() + 4 * n; }
    static size_t bytes_for(int64_t n) { return (size_t)n * 5 * sizeof(float4); }
    int alloc(int64_t nn)
    {
        n = nn;
        return mem.ensure(bytes_for(nn));
    }
    void place(int64_t nn, void *region)
    {
        n = nn;
        ext = static_cast<float4 *>(region);
    }
};

// Copies n x 4 floats (host or device, per flags) into a device array.
int upload4(float4 *dst, const float *src, int64_t n, unsigned flags, cudaStream_t st)
{
    const size_t nb = (size_t)n * sizeof(float4);
    CKR(cudaMemcpyAsync(dst, src, nb, (flags & BH_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice
                                                               : cudaMemcpyHostToDevice, st));
    return BH_OK;
}

int download4(float *dst, const float4 *src, int64_t n, unsigned flags, cudaStream_t st)
{
    const size_t nb = (size_t)n * sizeof(float4);
    CKR(cudaMemcpyAsync(dst, src, nb, (flags & BH_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice
                                                               : cudaMemcpyDeviceToHost, st));
    return BH_OK;
}

// ------------------------------------------------------- autotune cache

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, unsigned>, bh_tuning> g_tune_cache;

int log2_bucket(int64_t n)
{
    int b = 0;
    while ((1ll << (b + 1)) <= n) ++b;
    return b;
}

// ----------------------------------------------------------------- Forest

struct Forest {
    cudaStream_t st = nullptr;
    cudaStream_t user = nullptr;
    cudaEvent_t ev_sync = nullptr;
    cudaEvent_t ev_step = nullptr;  // end of a step enqueued by step_begin
    int dev = 0, nsm = 0;
    unsigned flags = 0;
    std::vector<SysState *> systems;
    std::vector<std::unique_ptr<SysState>> owned;

    std::vector<SysStatic> h_sys;
    std::vector<int4> h_chunks;
    std::vector<int> h_mode;
    int n_total = 0, nchunks = 0, nsys = 0;
    bool tables_dirty = true;

    DevBuf d_sys, d_dyn, d_chunks, d_mode, d_parts, key0, key1, val0, val1, rs_counts, scan_part,
        spos, ncount, noff, nodeW, nodeR, nodeD, nlist, nodeI, nodeQ, nodeB, nodeF, nodeDF, lidx,
        ldfs, sib_count, d_small, d_diag_parts, d_diag_out, d_counts, d_export;
    unsigned node_cap = 0;
    struct TileSet {
        DevBuf buf;
        int ntiles = 0;
        bool valid = false;
    } tiles[3];
    Small *h_small = nullptr;  // pinned mirror

    bool acc_valid = false;
    bool tree_valid = false;
    bh_tuning tune{1, 16, 0, 1, 90};

    cudaGraphExec_t gexec = nullptr;
    int g_nsteps = -1;
    unsigned g_cap = 0;
    bh_tuning g_tune{0, 0, 0, 0, 0};
    int g_ntotal = -1;
    bool g_prof = false;  // the graph carries phase events
    int g_sort_first = -1;

    // the short sort's first radix pass: the top three digits to start with;
    // a build that meets a longer run than the fixup sorts is redone with one
    // digit more, down to the full sort (0), which then stays
    int sort_first = 5;

    // first level of the fused deep centre-of-mass launch, chosen from the
    // previous build's level sizes (22 = none yet)
    int deep_cut = kNumLevels;
    // off where the set of systems changes between steps (the server): the
    // previous build then says little about the next one's level sizes
    bool adaptive_deep = true;
    bool do_walk = true;
    int64_t last_step_launches = 0;
    // phase profiling: events around the phases of each step, on st.  Steps
    // enqueued directly use ev_plain (recycled after each run); steps captured
    // in the graph use ev_graph (re-recorded by every replay).
    bool prof = false;
    bool capturing = false;
    std::vector<cudaEvent_t> ev_plain, ev_graph;
    size_t ev_plain_used = 0;
    std::vector<std::array<int, 5>> plain_marks, graph_marks;
    double prof_ms[BH_NPHASE] = {0, 0, 0};
    int64_t prof_nsteps = 0;
    int64_t launches = 0;

    ~Forest()
    {
        if (gexec) cudaGraphExecDestroy(gexec);
        for (cudaEvent_t e : ev_plain) cudaEventDestroy(e);
        for (cudaEvent_t e : ev_graph) cudaEventDestroy(e);
        if (ev_sync) cudaEventDestroy(ev_sync);
        if (ev_step) cudaEventDestroy(ev_step);
        if (h_small) cudaFreeHost(h_small);
        if (st) cudaStreamDestroy(st);
    }

    int init(void *user_stream, unsigned fl)
    {
        flags = fl;
        user = (cudaStream_t)user_stream;
        CKR(cudaGetDevice(&dev));
        CKR(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        CKR(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        prepare_sort_kernels();
        CKR(cudaEventCreateWithFlags(&ev_sync, cudaEventDisableTiming));
        CKR(cudaEventCreateWithFlags(&ev_step, cudaEventDisableTiming));
        CKR(cudaMallocHost(&h_small, sizeof(Small)));
        std::memset(h_small, 0, sizeof(Small));
        TRY(d_small.ensure(sizeof(Small)));
        CKR(cudaMemsetAsync(d_small.p, 0, sizeof(Small), st));
        return BH_OK;
    }

    // Orders this call's work after everything already queued on the
    // caller's stream (e.g. tensors the caller just wrote).
    int begin_call()
    {
        CKR(cudaEventRecord(ev_sync, user));
        CKR(cudaStreamWaitEvent(st, ev_sync, 0));
        return BH_OK;
    }

    int sync()
    {
        CKR(cudaStreamSynchronize(st));
        return BH_OK;
    }

    Small *small() const { return d_small.as<Small>(); }

    BuildBufs bufs() const
    {
        BuildBufs b;
        b.chunks = d_chunks.as<int4>();
        b.nchunks = nchunks;
        b.sys = d_sys.as<SysStatic>();
        b.dyn = d_dyn.as<SysDyn>();
        b.nsys = nsys;
        b.mode = d_mode.as<int>();
        b.parts = d_parts.as<ChunkPart>();
        b.key0 = key0.as<uint64_t>();
        b.key1 = key1.as<uint64_t>();
        b.val0 = val0.as<uint32_t>();
        b.val1 = val1.as<uint32_t>();
        b.rs_counts = rs_counts.as<uint32_t>();
        b.scan_part = scan_part.as<uint32_t>();
        b.spos = spos.as<float4>();
        b.ncount = ncount.as<uint32_t>();
        b.noff = noff.as<uint32_t>();
        b.nodeW = nodeW.as<WNode>();
        b.nodeR = nodeR.as<int4>();
        b.nodeD = nodeD.as<double4_32a>();
        b.nlist = nlist.as<uint32_t>();
        b.nodeI = quad() ? nodeI.as<double>() : nullptr;
        b.nodeQ = quad() ? nodeQ.as<float4>() : nullptr;
        b.nodeB = bmax() ? nodeB.as<double>() : nullptr;
        const bool sib = sib_walk() && nodeF.p;
        b.nodeF = sib ? nodeF.as<WNode>() : nullptr;
        b.nodeDF = sib ? nodeDF.as<double4_32a>() : nullptr;
        b.lidx = sib ? lidx.as<uint32_t>() : nullptr;
        b.ldfs = sib ? ldfs.as<uint32_t>() : nullptr;
        b.sib_count = sib ? sib_count.as<uint32_t>() : nullptr;
        b.node_cap = node_cap;
        b.small = small();
        b.n_total = n_total;
        b.nsm = nsm;
        b.deep_cut = deep_cut;
        b.sort_first = sort_first;
        return b;
    }

    int ensure_nodes(size_t cap)
    {
        if (cap <= node_cap && nodeW.p) return BH_OK;
        TRY(nodeW.ensure(cap * sizeof(WNode)));
        TRY(nodeR.ensure(cap * sizeof(int4)));
        TRY(nodeD.ensure(cap * sizeof(double4_32a)));
        TRY(nlist.ensure(cap * sizeof(uint32_t)));
        if (quad()) {
            TRY(nodeI.ensure(cap * 6 * sizeof(double)));
            TRY(nodeQ.ensure(cap * 2 * sizeof(float4)));
        }
        if (bmax()) TRY(nodeB.ensure(cap * sizeof(double)));
        node_cap = (unsigned)cap;
        invalidate_graph();
        return BH_OK;
    }

    // Buffers of the sibling-order walk, sized for the node capacity (the
    // child-count scan runs over all of it, so its partials too); allocated
    // only while that walk is the tuned shape, and never during a capture.
    int ensure_sib_bufs()
    {
        if (!sib_walk()) return BH_OK;
        const size_t cap = node_cap;
        const size_t want[6] = {cap * sizeof(WNode), cap * sizeof(double4_32a), cap * 4, cap * 4,
                                cap * 4, ((cap + kScanTile - 1) / kScanTile + 1) * 4};
        DevBuf *bufs4[6] = {&nodeF, &nodeDF, &lidx, &ldfs, &sib_count, &scan_part};
        bool moved = false;
        for (int q = 0; q < 6; ++q) {
            if (bufs4[q]->p && bufs4[q]->bytes >= want[q]) continue;
            TRY(bufs4[q]->ensure(want[q]));
            moved = true;
        }
        if (moved) invalidate_graph();
        return BH_OK;
    }

    void invalidate_graph()
    {
        if (gexec) cudaGraphExecDestroy(gexec);
        gexec = nullptr;
        g_nsteps = -1;
    }

    // Builds the system / chunk tables from `systems` and sizes the scratch.
    int setup()
    {
        nsys = (int)systems.size();
        h_sys.assign(nsys, SysStatic{});
        h_chunks.clear();
        int64_t start = 0;
        for (int s = 0; s < nsys; ++s) {
            SysState *S = systems[s];
            SysStatic &d = h_sys[s];
            d.pos = S->pos(); d.vel = S->vel(); d.acc = S->acc(); d.bpos = S->bpos(); d.bvel = S->bvel();
            d.start = (int)start;
            d.n = (int)S->n;
            d.chunk0 = (int)h_chunks.size();
            for (int64_t c = 0; c < S->n; c += kChunk)
                h_chunks.push_back(make_int4(s, (int)(start + c), (int)std::min<int64_t>(kChunk, S->n - c), 0));
            d.nchunk = (int)h_chunks.size() - d.chunk0;
            d.eps2 = (float)(S->eps * S->eps);
            d.G = (float)S->G;
            d.inv_theta2 = S->theta > 0.0 ? (float)(1.0 / (S->theta * S->theta)) : INFINITY;
            d.half_dt = (float)(0.5 * S->dt);
            d.dt = (float)S->dt;
            d.flags = 0;
            d.theta2 = S->theta * S->theta;
            start += S->n;
            if (start > (int64_t)INT_MAX / 2) return fail(BH_ERR_INVALID, "too many particles (limit 2^30)");
        }
        n_total = (int)start;
        nchunks = (int)h_chunks.size();
        if (n_total < 1) return fail(BH_ERR_INVALID, "no particles");
        h_mode.assign(nsys, MODE_KDK);
        TRY(d_sys.ensure(sizeof(SysStatic) * nsys));
        TRY(d_dyn.ensure(sizeof(SysDyn) * nsys));
        TRY(d_mode.ensure(sizeof(int) * nsys));
        TRY(d_chunks.ensure(sizeof(int4) * nchunks));
        TRY(d_parts.ensure(sizeof(ChunkPart) * nchunks));
        TRY(d_diag_parts.ensure(sizeof(DiagPart) * nchunks));
        TRY(d_diag_out.ensure(sizeof(double) * 8 * nsys));
        CKR(cudaMemcpyAsync(d_sys.p, h_sys.data(), sizeof(SysStatic) * nsys, cudaMemcpyHostToDevice, st));
        CKR(cudaMemcpyAsync(d_chunks.p, h_chunks.data(), sizeof(int4) * nchunks, cudaMemcpyHostToDevice, st));
        CKR(cudaMemcpyAsync(d_mode.p, h_mode.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, st));
        const size_t N = (size_t)n_total;
        bool moved = false;
        auto grow = [&](DevBuf &b, size_t nb) -> int {
            void *old = b.p;
            int rc = b.ensure(nb);
            if (b.p != old) moved = true;
            return rc;
        };
        TRY(grow(key0, N * 8));
        TRY(grow(key1, N * 8));
        TRY(grow(val0, N * 4));
        TRY(grow(val1, N * 4));
        TRY(grow(spos, N * 16));
        TRY(grow(ncount, (N + 1) * 4));
        TRY(grow(noff, (N + 1) * 4));
        const size_t ncounts = (size_t)kRadixBins * nchunks;
        TRY(grow(rs_counts, 2 * ncounts * 4));
        const size_t scan_n = std::max(ncounts, N + 1);
        TRY(grow(scan_part, ((scan_n + kScanTile - 1) / kScanTile + 1) * 4));
        TRY(ensure_nodes(2 * N + 1024));
        for (auto &t : tiles) t.valid = false;
        if (moved) invalidate_graph();
        tables_dirty = false;
        tree_valid = false;
        return BH_OK;
    }

    int upload_sys_table()
    {
        CKR(cudaMemcpyAsync(d_sys.p, h_sys.data(), sizeof(SysStatic) * nsys, cudaMemcpyHostToDevice, st));
        return BH_OK;
    }

    int set_dt(double dt)
    {
        bool changed = false;
        for (int s = 0; s < nsys; ++s) {
            const float hd = (float)(0.5 * dt), d = (float)dt;
            if (h_sys[s].half_dt != hd || h_sys[s].dt != d) changed = true;
            h_sys[s].half_dt = hd;
            h_sys[s].dt = d;
            systems[s]->dt = dt;
        }
        if (changed) TRY(upload_sys_table());
        return BH_OK;
    }

    int set_modes(const std::vector<int> &m)
    {
        if (m == h_mode) return BH_OK;
        h_mode = m;
        CKR(cudaMemcpyAsync(d_mode.p, h_mode.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, st));
        // the copy reads pageable memory: make sure it has been consumed
        CKR(cudaStreamSynchronize(st));
        return BH_OK;
    }

    int set_all_modes(int m) { return set_modes(std::vector<int>(nsys, m)); }

    int tile_index(int ppl) const { return ppl == 1 ? 0 : (ppl == 2 ? 1 : 2); }

    int ensure_tiles(int ppl)
    {
        TileSet &T = tiles[tile_index(ppl)];
        if (T.valid) return BH_OK;
        std::vector<Tile> t;
        const int sz = 32 * ppl;
        for (int s = 0; s < nsys; ++s) {
            const SysStatic &S = h_sys[s];
            for (int o = 0; o < S.n; o += sz) t.push_back(Tile{S.start + o, std::min(sz, S.n - o), s, 0});
        }
        TRY(T.buf.ensure(sizeof(Tile) * t.size()));
        CKR(cudaMemcpyAsync(T.buf.p, t.data(), sizeof(Tile) * t.size(), cudaMemcpyHostToDevice, st));
        CKR(cudaStreamSynchronize(st));
        T.ntiles = (int)t.size();
        T.valid = true;
        return BH_OK;
    }

    WalkArgs walk_args(int ppl, uint32_t *counts) const
    {
        WalkArgs a;
        a.nodeW = nodeW.as<WNode>();
        a.nodeQ = quad() ? nodeQ.as<float4>() : nullptr;
        a.nodeR = nodeR.as<int4>();
        a.nodeD = nodeD.as<double4_32a>();
        a.nodeB = bmax() ? nodeB.as<double>() : nullptr;
        // the sibling-order walk reads the sibling-order copies in their place
        if (sib_walk() && nodeF.p) {
            a.nodeW = nodeF.as<WNode>();
            a.nodeD = nodeDF.as<double4_32a>();
        }
        a.dyn = d_dyn.as<SysDyn>();
        a.spos = spos.as<float4>();
        a.sid = val0.as<uint32_t>();
        a.noff = noff.as<uint32_t>();
        const TileSet &T = tiles[tile_index(ppl)];
        a.tiles = T.buf.as<Tile>();
        a.ntiles = T.ntiles;
        a.sys = d_sys.as<SysStatic>();
        a.mode = d_mode.as<int>();
        a.small = small();
        a.counts = counts;
        a.static_share = tune.static_share;
        a.nsm = nsm;
        return a;
    }

    // BH_OPEN_INSIDE and BH_QUADRUPOLE fix the shape to one particle per lane
    WalkShape shape() const { return shape_of(tune); }
    WalkShape shape_of(const bh_tuning &t) const
    {
        if (fixed_shape())
            return WalkShape{1, t.warps_per_block, t.blocks_per_sm, 1, open_inside(), quad(), false};
        return WalkShape{t.ppl, t.warps_per_block, t.blocks_per_sm, walk_group(t.group), false,
                         false, all_soft()};
    }
    // the split walk (group 0) recognises its top-level nodes by their
    // threshold, and the sibling-order walk forms it from the level: both need
    // it to be a function of the level alone, which under the b_max rule it
    // is not, so there they run as group 1
    int walk_group(int g) const
    {
        return fixed_shape() || (bmax() && (g == 0 || g == BH_GROUP_SIBLINGS)) ? 1 : g;
    }
    bool sib_walk() const { return shape().group == BH_GROUP_SIBLINGS; }
    // every system of the current tables has a positive softening length
    bool all_soft() const
    {
        for (const SysStatic &d : h_sys)
            if (!(d.eps2 > 0.f)) return false;
        return !h_sys.empty();
    }
    bool open_inside() const { return (flags & BH_OPEN_INSIDE) != 0; }
    bool quad() const { return (flags & BH_QUADRUPOLE) != 0; }
    bool bmax() const { return (flags & BH_OPEN_BMAX) != 0; }
    bool fixed_shape() const { return open_inside() || quad(); }
    bool kahan() const { return !(flags & BH_NO_KAHAN); }
    bool pot() const { return (flags & BH_POTENTIAL) != 0; }

    int mark()
    {
        if (!prof) return -1;
        std::vector<cudaEvent_t> &pool = capturing ? ev_graph : ev_plain;
        const size_t idx = capturing ? ev_graph_next++ : ev_plain_used++;
        while (pool.size() <= idx) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return -1;
            pool.push_back(e);
        }
        // inside a capture only an external record becomes a graph node that
        // re-records the event on every replay
        if (capturing) cudaEventRecordWithFlags(pool[idx], st, cudaEventRecordExternal);
        else cudaEventRecord(pool[idx], st);
        return (int)idx;
    }

    size_t ev_graph_next = 0;

    // Adds the device time of the recorded steps' phases to prof_ms.
    void accumulate(const std::vector<std::array<int, 5>> &marks, const std::vector<cudaEvent_t> &pool)
    {
        for (const auto &m : marks) {
            if (m[0] < 0 || m[4] < 0) continue;
            float a = 0, b2 = 0, c = 0, d = 0;
            cudaEventElapsedTime(&a, pool[m[0]], pool[m[1]]);
            cudaEventElapsedTime(&b2, pool[m[1]], pool[m[2]]);
            cudaEventElapsedTime(&c, pool[m[2]], pool[m[3]]);
            cudaEventElapsedTime(&d, pool[m[3]], pool[m[4]]);
            prof_ms[0] += a + d;
            prof_ms[1] += b2;
            prof_ms[2] += c;
            prof_nsteps += 1;
        }
    }

    void reset_step_counters()
    {
        const size_t off = offsetof(Small, queue);
        const size_t len = offsetof(Small, level_off) - off;
        cudaMemsetAsync(reinterpret_cast<char *>(small()) + off, 0, len, st);
    }

    // Enqueues one step (per-system mode from d_mode).
    int enqueue_step()
    {
        TRY(ensure_tiles(tune.ppl));
        g_launches = 0;
        const BuildBufs b = bufs();
        std::array<int, 5> m;
        reset_step_counters();
        m[0] = mark();
        launch_kick_drift_bbox(b, st);
        m[1] = mark();
        launch_keys(b, st);
        launch_sort(b, st);
        launch_permute(b, st);
        launch_topology(b, st);
        launch_com(b, st);
        if (sib_walk()) {
            if (!b.nodeF) return fail(BH_ERR_STATE, "sibling-order buffers missing");
            launch_sibling_order(b, st);
        }
        m[2] = mark();
        if (do_walk &&
            launch_walk(walk_args(tune.ppl, nullptr), shape(), kahan(), pot(), false, nsm, st) < 0)
            return fail(BH_ERR_INVALID, "unsupported walk shape");
        m[3] = mark();
        launch_kick(b, st);
        m[4] = mark();
        if (prof) (capturing ? graph_marks : plain_marks).push_back(m);
        last_step_launches = g_launches;
        launches += g_launches;
        CKR(cudaGetLastError());
        return BH_OK;
    }

    int read_small()
    {
        CKR(cudaMemcpyAsync(h_small, d_small.p, sizeof(Small), cudaMemcpyDeviceToHost, st));
        CKR(cudaStreamSynchronize(st));
        return BH_OK;
    }

    int clear_status()
    {
        CKR(cudaMemsetAsync(d_small.p, 0, offsetof(Small, wstats), st));
        return BH_OK;
    }

    int capture_graph(int nsteps)
    {
        invalidate_graph();
        cudaGraph_t g = nullptr;
        graph_marks.clear();
        ev_graph_next = 0;
        capturing = true;
        CKR(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        int rc = BH_OK;
        for (int k = 0; k < nsteps && rc == BH_OK; ++k) rc = enqueue_step();
        cudaError_t e = cudaStreamEndCapture(st, &g);
        capturing = false;
        g_prof = prof;
        if (rc != BH_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return fail(BH_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            gexec = nullptr;
            return fail(BH_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        }
        g_nsteps = nsteps;
        g_cap = node_cap;
        g_tune = tune;
        g_sort_first = sort_first;
        g_ntotal = n_total;
        return BH_OK;
    }

    // Runs nsteps steps with the current modes; handles node-capacity
    // overflow by rolling back, growing and retrying.
    int run(int nsteps, bool graph)
    {
        int remaining = nsteps;
        for (int attempt = 0; remaining > 0; ++attempt) {
            // each retry grows the node buffer or adds a sort digit (at most 5)
            if (attempt > 16) return fail(BH_ERR_CAPACITY, "node buffer kept overflowing");
            TRY(launch_steps(remaining, graph));
            TRY(read_small());
            TRY(settle(remaining, graph));
        }
        tree_valid = true;
        return BH_OK;
    }

    // Enqueues `count` steps (from the captured graph or launched directly).
    int launch_steps(int count, bool graph)
    {
        TRY(clear_status());
        TRY(ensure_tiles(tune.ppl));
        TRY(ensure_sib_bufs());
        if (graph) {
            walk_max_blocks_per_sm(shape(), kahan(), pot());  // occupancy query outside capture
            if (!gexec || g_nsteps != count || g_cap != node_cap || g_ntotal != n_total ||
                g_sort_first != sort_first || std::memcmp(&g_tune, &tune, sizeof tune) != 0 ||
                (prof && !g_prof))
                TRY(capture_graph(count));
            CKR(cudaGraphLaunch(gexec, st));
            launches += (int64_t)count * steps_launches();
        } else {
            for (int k = 0; k < count; ++k) TRY(enqueue_step());
        }
        return BH_OK;
    }

    // After the launched steps have finished and h_small holds the device
    // status: remaining = 0 when they all succeeded; after a node-buffer
    // overflow or a sort run too long for the short sort, the failed step is
    // rolled back, the buffer grown (or a sort digit added) and remaining set
    // to the steps still to do.
    int settle(int &remaining, bool graph)
    {
        choose_deep_cut();
        if (prof) {
            if (graph) {
                if (g_prof) accumulate(graph_marks, ev_graph);
            } else {
                accumulate(plain_marks, ev_plain);
            }
            plain_marks.clear();
            ev_plain_used = 0;
        }
        const Small &h = *h_small;
        if (h.status == ST_OK) {
            remaining = 0;
            return BH_OK;
        }
        if (h.status == ST_SORT_LONG) {  // redo with one more digit, from here on
            const int done = (int)h.steps_done;
            launch_restore(bufs(), st);
            launches += 1;
            sort_first = sort_first > 0 ? sort_first - 1 : 0;
            remaining -= done;
            tree_valid = false;
            return BH_OK;
        }
        if (h.status == ST_CAPACITY) {
            const int done = (int)h.steps_done;
            launch_restore(bufs(), st);
            launches += 1;
            const size_t want = (size_t)h.needed + h.needed / 4 + 1024;
            TRY(ensure_nodes(want));
            remaining -= done;
            tree_valid = false;
            return BH_OK;
        }
        if (h.status == ST_WALK_LIMIT)
            return fail(BH_ERR_CUDA, "walk stopped on a corrupt tree (skip pointer not advancing)");
        return fail(BH_ERR_CUDA, "device status " + std::to_string(h.status));
    }

    // One step without waiting for it (the server overlaps its host work and
    // copies with the step): step_begin enqueues it and the read-back of the
    // device status; step_end waits for both and then behaves like run(1).
    int step_begin()
    {
        TRY(launch_steps(1, false));
        CKR(cudaMemcpyAsync(h_small, d_small.p, sizeof(Small), cudaMemcpyDeviceToHost, st));
        CKR(cudaEventRecord(ev_step, st));
        return BH_OK;
    }

    int step_end()
    {
        CKR(cudaEventSynchronize(ev_step));
        int remaining = 1;
        TRY(settle(remaining, false));
        if (remaining > 0) return run(remaining, false);
        tree_valid = true;
        return BH_OK;
    }

    // Sizes every buffer for up to n_max particles in up to nsys_max systems,
    // so that setup() for any set of systems within those limits allocates
    // nothing (only a node-buffer overflow still grows the node arrays).
    int reserve(int64_t n_max, int nsys_max)
    {
        const size_t N = (size_t)n_max;
        const size_t chunks = N / kChunk + (size_t)nsys_max;
        const size_t ntiles = N / 32 + (size_t)nsys_max;
        TRY(d_sys.ensure(sizeof(SysStatic) * nsys_max));
        TRY(d_dyn.ensure(sizeof(SysDyn) * nsys_max));
        TRY(d_mode.ensure(sizeof(int) * nsys_max));
        TRY(d_diag_out.ensure(sizeof(double) * 8 * nsys_max));
        TRY(d_chunks.ensure(sizeof(int4) * chunks));
        TRY(d_parts.ensure(sizeof(ChunkPart) * chunks));
        TRY(d_diag_parts.ensure(sizeof(DiagPart) * chunks));
        TRY(key0.ensure(N * 8));
        TRY(key1.ensure(N * 8));
        TRY(val0.ensure(N * 4));
        TRY(val1.ensure(N * 4));
        TRY(spos.ensure(N * 16));
        TRY(ncount.ensure((N + 1) * 4));
        TRY(noff.ensure((N + 1) * 4));
        const size_t ncounts = (size_t)kRadixBins * chunks;
        TRY(rs_counts.ensure(2 * ncounts * 4));
        const size_t scan_n = std::max(ncounts, N + 1);
        TRY(scan_part.ensure(((scan_n + kScanTile - 1) / kScanTile + 1) * 4));
        TRY(ensure_nodes(2 * N + 1024));
        for (auto &t : tiles) TRY(t.buf.ensure(sizeof(Tile) * ntiles));
        return BH_OK;
    }

    // Deep levels whose nodes sum to at most kDeepNodes go to one launch.
    void choose_deep_cut()
    {
        constexpr unsigned kDeepNodes = 512;
        if (!adaptive_deep) return;
        unsigned sum = 0;
        int cut = kNumLevels;
        for (int l = kLevels; l >= 1; --l) {
            sum += h_small->level_cnt[l];
            if (sum > kDeepNodes) break;
            cut = l;
        }
        deep_cut = cut;
    }

    // kernels per step, as counted by the launchers when the step was enqueued
    int64_t steps_launches() const { return last_step_launches; }

    int compute_accel()
    {
        TRY(set_all_modes(MODE_ACCEL));
        TRY(run(1, false));
        acc_valid = true;
        return BH_OK;
    }

    // Tree only (no walk): positions, and so any stored acceleration, unchanged.
    int build_only()
    {
        TRY(set_all_modes(MODE_ACCEL));
        do_walk = false;
        const int rc = run(1, false);
        do_walk = true;
        return rc;
    }

    int step(int nsteps, bool graph)
    {
        if (!acc_valid) TRY(compute_accel());
        TRY(set_all_modes(MODE_KDK));
        return run(nsteps, graph);
    }

    int ensure_tree()
    {
        if (tree_valid) return BH_OK;
        return compute_accel();
    }

    int autotune(bh_tuning *best)
    {
        double th = 0;
        for (auto *s : systems) th += s->theta;
        th /= std::max(1, nsys);
        const auto key = std::make_tuple(dev, log2_bucket(n_total), (int)std::lround(th * 20), nsys > 1 ? 1 : 0,
                                         flags & (BH_POTENTIAL | BH_NO_KAHAN | BH_OPEN_INSIDE |
                                                  BH_QUADRUPOLE | BH_OPEN_BMAX));
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) {
                tune = it->second;
                if (best) *best = tune;
                return BH_OK;
            }
        }
        TRY(ensure_tree());
        // (group, particles per lane) candidates x warps per block
        // (the interaction-list walk is left out: measured 2-2.5x slower than
        // the fused walks on every workload tried, it would only lengthen tuning)
        // (the sibling-order walk is left out too: slower than one lane per
        // particle in depth-first order on every workload measured, and its
        // copy adds build time the walk-only timing here would not see)
        const int shapes[10][2] = {{0, 1}, {1, 1}, {1, 2}, {1, 4}, {2, 1}, {4, 1}, {8, 1}, {32, 1},
                                   {32, 2}, {32, 4}};
        // (14: three blocks of 14 warps, 42 per SM, fewer walks sharing L1,
        // measured ~0.7% faster than 48 on the 1M cube at theta 0.5 and 0.7)
        const int warps[3] = {8, 14, 16};
        cudaEvent_t e0, e1;
        CKR(cudaEventCreate(&e0));
        CKR(cudaEventCreate(&e1));
        // static shares: none (forests of uneven systems), 90 (one system: the
        // best measured with taking from the SMs' neighbouring ranges), 100
        const int shares[3] = {0, 90, 100};
        const bh_tuning saved = tune;
        // best walk time of `reps` launches (the first is not counted)
        auto time_walk = [&](const bh_tuning &t, int reps) -> float {
            tune = t;  // walk_args reads the static share from tune
            const WalkShape sh = shape_of(t);
            float ms_best = 1e30f;
            for (int rep = 0; rep < reps; ++rep) {
                reset_step_counters();
                cudaEventRecord(e0, st);
                launch_walk(walk_args(t.ppl, nullptr), sh, kahan(), pot(), false, nsm, st);
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) != cudaSuccess) return 1e30f;
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0 && ms < ms_best) ms_best = ms;
            }
            return ms_best;
        };
        // round one: every candidate, two timed launches each
        std::vector<std::pair<float, bh_tuning>> timed;
        for (const auto &gp : shapes) {
            const int g = gp[0], p = gp[1];
            TRY(ensure_tiles(p));
            for (int w : warps) {
                for (int share : shares) {
                    bh_tuning t{p, w, 0, g, share};
                    if (fixed_shape() && (g != 1 || p != 1)) continue;
                    if (bmax() && g == 0) continue;
                    if (walk_max_blocks_per_sm(shape_of(t), kahan(), pot()) <= 0) continue;
                    timed.push_back({time_walk(t, 3), t});
                }
            }
        }
        // round two: the four fastest again, six timed launches each (shapes
        // a few per cent apart are otherwise picked by timing noise)
        std::sort(timed.begin(), timed.end(), [](const std::pair<float, bh_tuning> &x,
                                                 const std::pair<float, bh_tuning> &y) {
            return x.first < y.first;
        });
        float best_ms = 1e30f;
        bh_tuning pick = saved;
        for (size_t k = 0; k < timed.size() && k < 4; ++k) {
            const float ms = time_walk(timed[k].second, 7);
            if (ms < best_ms) {
                best_ms = ms;
                pick = timed[k].second;
            }
        }
        tune = saved;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        CKR(cudaGetLastError());
        tune = pick;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune_cache[key] = pick;
        }
        if (best) *best = pick;
        return BH_OK;
    }

    int set_tuning(const bh_tuning *t)
    {
        if (!t || (t->ppl != 1 && t->ppl != 2 && t->ppl != 4) || t->warps_per_block < 1 ||
            t->warps_per_block > 32 || t->blocks_per_sm < 0 ||
            t->warps_per_block > 16 ||
            (t->group != 0 && t->group != 1 && t->group != 2 && t->group != 4 && t->group != 8 &&
             t->group != 32 && t->group != BH_GROUP_LIST && t->group != BH_GROUP_SIBLINGS) ||
            t->static_share < 0 || t->static_share > 100 ||
            (t->group != 32 && t->group != 1 && t->ppl == 4) ||
            ((t->group == 2 || t->group == 0 || t->group == BH_GROUP_LIST ||
              t->group == BH_GROUP_SIBLINGS) && t->ppl != 1))
            return fail(BH_ERR_INVALID, "bad tuning (group 1 or 32 with ppl 1/2/4, group 4/8 with "
                                        "ppl 1/2, group 2, 0, BH_GROUP_LIST or BH_GROUP_SIBLINGS "
                                        "with ppl 1; warps 1..16; static_share 0..100; "
                                        "blocks_per_sm >= 0)");
        // the shape as it would be launched (BH_OPEN_INSIDE: one particle per lane)
        const WalkShape sh = shape_of(*t);
        if (walk_max_blocks_per_sm(sh, kahan(), pot()) <= 0)
            return fail(BH_ERR_INVALID, "walk shape does not fit on an SM");
        tune = *t;
        return BH_OK;
    }

    int diagnostics(std::vector<double> &out)
    {
        launch_diagnostics(bufs(), d_diag_parts.as<DiagPart>(), d_diag_out.as<double>(), st);
        launches += 2;
        out.assign(8 * nsys, 0.0);
        CKR(cudaMemcpyAsync(out.data(), d_diag_out.p, sizeof(double) * 8 * nsys, cudaMemcpyDeviceToHost, st));
        TRY(sync());
        if (!pot())
            for (int s = 0; s < nsys; ++s) out[8 * s + 1] = NAN;
        return BH_OK;
    }

    int interaction_count(int sys, uint32_t *counts, uint64_t *total)
    {
        TRY(ensure_tree());
        TRY(d_counts.ensure(sizeof(uint32_t) * (size_t)n_total));
        TRY(ensure_tiles(1));
        TRY(clear_status());
        reset_step_counters();
        WalkShape sh{1, 8, 0, walk_group(tune.group), open_inside(), quad(), false};
        if (sh.group == BH_GROUP_SIBLINGS) {  // its copy of the current tree
            TRY(ensure_sib_bufs());
            launch_sibling_order(bufs(), st);
            launches += 3;
        }
        CKR(cudaMemsetAsync(small()->wstats, 0, sizeof(small()->wstats), st));
        launch_walk(walk_args(1, d_counts.as<uint32_t>()), sh, true, false, true, nsm, st);
        launches += 1;
        const SysStatic &S = h_sys[sys];
        std::vector<uint32_t> h((size_t)S.n);
        CKR(cudaMemcpyAsync(h.data(), d_counts.as<uint32_t>() + S.start, sizeof(uint32_t) * S.n,
                            cudaMemcpyDeviceToHost, st));
        TRY(read_small());
        if (h_small->status != ST_OK) return fail(BH_ERR_CUDA, "counting walk failed");
        uint64_t t = 0;
        for (uint32_t c : h) t += c;
        if (counts) std::memcpy(counts, h.data(), sizeof(uint32_t) * S.n);
        if (total) *total = t;
        return BH_OK;
    }

    int export_tree(int sys, uint64_t *keys, uint32_t *order, bh_node *nodes, float *com_m,
                    int64_t node_cap_out, int64_t *n_nodes, float *cube)
    {
        TRY(ensure_tree());
        const SysStatic &S = h_sys[sys];
        uint32_t n01[2];
        CKR(cudaMemcpyAsync(&n01[0], noff.as<uint32_t>() + S.start, 4, cudaMemcpyDeviceToHost, st));
        CKR(cudaMemcpyAsync(&n01[1], noff.as<uint32_t>() + S.start + S.n, 4, cudaMemcpyDeviceToHost, st));
        TRY(sync());
        const int64_t M = (int64_t)n01[1] - n01[0];
        if (n_nodes) *n_nodes = M;
        if ((nodes || com_m) && M > node_cap_out)
            return fail(BH_ERR_INVALID, "node_cap too small: need " + std::to_string(M));
        const size_t nb_nodes = sizeof(bh_node) * M, nb_com = sizeof(float4) * M, nb_ord = 4 * (size_t)S.n;
        TRY(d_export.ensure(nb_nodes + nb_com + nb_ord + 64));
        char *base = d_export.as<char>();
        bh_node *dn = reinterpret_cast<bh_node *>(base);
        float4 *dc = reinterpret_cast<float4 *>(base + ((nb_nodes + 15) & ~size_t(15)));
        uint32_t *dord = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(dc) + nb_com);
        launch_export(bufs(), sys, dn, dc, dord, st);
        launches += 1;
        if (nodes) CKR(cudaMemcpyAsync(nodes, dn, nb_nodes, cudaMemcpyDeviceToHost, st));
        if (com_m) CKR(cudaMemcpyAsync(com_m, dc, nb_com, cudaMemcpyDeviceToHost, st));
        if (order) CKR(cudaMemcpyAsync(order, dord, nb_ord, cudaMemcpyDeviceToHost, st));
        if (keys) CKR(cudaMemcpyAsync(keys, key0.as<uint64_t>() + S.start, 8 * (size_t)S.n, cudaMemcpyDeviceToHost, st));
        if (cube) {
            SysDyn d;
            CKR(cudaMemcpyAsync(&d, d_dyn.as<SysDyn>() + sys, sizeof d, cudaMemcpyDeviceToHost, st));
            TRY(sync());
            cube[0] = d.lo[0]; cube[1] = d.lo[1]; cube[2] = d.lo[2]; cube[3] = d.side;
        }
        TRY(sync());
        return BH_OK;
    }

    int validate_device()
    {
        TRY(clear_status());
        launch_validate(bufs(), st);
        launches += 1;
        TRY(read_small());
        if (h_small->status == ST_BAD_INPUT) {
            clear_status();
            return fail(BH_ERR_INVALID, "non-finite coordinate or non-positive mass in device input");
        }
        return BH_OK;
    }

    void profile_begin()
    {
        prof = true;
        plain_marks.clear();
        ev_plain_used = 0;
        for (int k = 0; k < BH_NPHASE; ++k) prof_ms[k] = 0;
        prof_nsteps = 0;
        launches = 0;
        if (gexec && !g_prof) invalidate_graph();  // recapture with the events
    }

    int profile_end(double *phase_ms, int64_t *steps, int64_t *nl)
    {
        TRY(sync());
        accumulate(plain_marks, ev_plain);
        plain_marks.clear();
        ev_plain_used = 0;
        if (phase_ms) for (int k = 0; k < BH_NPHASE; ++k) phase_ms[k] = prof_ms[k];
        if (steps) *steps = prof_nsteps;
        if (nl) *nl = launches;
        prof = false;
        return BH_OK;
    }
};

}  // namespace

// ======================================================================
//                               C ABI
// ======================================================================

struct bh_system {
    Forest f;
    bh_params p;
};

struct bh_forest {
    Forest f;
};

extern "C" {

const char *bh_last_error(void) { return g_err.c_str(); }

const char *bh_version(void) { return "bh-gb300 1.0 (sm_103a)"; }

int bh_params_default(bh_params *p)
{
    if (!p) return fail(BH_ERR_INVALID, "null params");
    p->G = 1.0;
    p->eps = 0.01;
    p->theta = 0.5;
    p->max_depth = BH_MAX_DEPTH;
    p->leaf_cap = 1;
    p->flags = 0;
    return BH_OK;
}

static int check_bh_params(const bh_params *p)
{
    if (!p) return fail(BH_ERR_INVALID, "null params");
    TRY(check_params(p->G, p->eps, p->theta));
    if (p->max_depth != BH_MAX_DEPTH) return fail(BH_ERR_INVALID, "max_depth must be 21");
    if (p->leaf_cap != 1) return fail(BH_ERR_INVALID, "leaf_cap must be 1");
    if (p->flags &
        ~(BH_POTENTIAL | BH_NO_KAHAN | BH_OPEN_INSIDE | BH_QUADRUPOLE | BH_OPEN_BMAX))
        return fail(BH_ERR_INVALID, "unknown params flags");
    if ((p->flags & BH_QUADRUPOLE) && (p->flags & BH_NO_KAHAN))
        return fail(BH_ERR_INVALID, "BH_QUADRUPOLE needs Kahan sums");
    return BH_OK;
}

static int load_state(Forest &f, SysState &S, const float *pm, const float *vel, unsigned flags)
{
    if (!(flags & BH_DEVICE_PTRS) && !finite_state(S.n, pm, vel))
        return fail(BH_ERR_INVALID, "non-finite coordinate or non-positive mass");
    TRY(upload4(S.pos(), pm, S.n, flags, f.st));
    if (vel) TRY(upload4(S.vel(), vel, S.n, flags, f.st));
    else CKR(cudaMemsetAsync(S.vel(), 0, (size_t)S.n * sizeof(float4), f.st));
    CKR(cudaMemsetAsync(S.acc(), 0, (size_t)S.n * sizeof(float4), f.st));
    return BH_OK;
}

int bh_create(bh_system **out, const bh_params *p, int64_t n, const float *pos_mass,
              const float *vel, void *stream, unsigned flags)
{
    if (!out) return fail(BH_ERR_INVALID, "null out");
    *out = nullptr;
    TRY(check_bh_params(p));
    if (n < 1 || n > (1ll << 30)) return fail(BH_ERR_INVALID, "n must be in [1, 2^30]");
    if (!pos_mass) return fail(BH_ERR_INVALID, "null pos_mass");
    if (flags & ~BH_DEVICE_PTRS) return fail(BH_ERR_INVALID, "unknown flags");
    std::unique_ptr<bh_system> s(new (std::nothrow) bh_system);
    if (!s) return fail(BH_ERR_OOM, "host allocation failed");
    s->p = *p;
    Forest &f = s->f;
    TRY(f.init(stream, p->flags));
    TRY(f.begin_call());
    auto st = std::make_unique<SysState>();
    st->G = p->G; st->eps = p->eps; st->theta = p->theta;
    TRY(st->alloc(n));
    TRY(load_state(f, *st, pos_mass, vel, flags));
    f.systems.push_back(st.get());
    f.owned.push_back(std::move(st));
    TRY(f.setup());
    if (flags & BH_DEVICE_PTRS) TRY(f.validate_device());
    TRY(f.sync());
    *out = s.release();
    return BH_OK;
}

int bh_destroy(bh_system *s)
{
    if (!s) return BH_OK;
    s->f.sync();
    delete s;
    return BH_OK;
}

int bh_set_state(bh_system *s, const float *pos_mass, const float *vel, const float *acc,
                 unsigned flags)
{
    if (!s || !pos_mass) return fail(BH_ERR_INVALID, "null argument");
    if (flags & ~BH_DEVICE_PTRS) return fail(BH_ERR_INVALID, "unknown flags");
    TRY(s->f.begin_call());
    Forest &f = s->f;
    SysState &S = *f.systems[0];
    // stage into the step-backup arrays (and the accelerations into the
    // sorted-position scratch, which the next build rewrites before any use)
    // and check there, so a rejected state leaves the system as it was
    TRY(upload4(S.bpos(), pos_mass, S.n, flags, f.st));
    if (vel) TRY(upload4(S.bvel(), vel, S.n, flags, f.st));
    float4 *acc_stage = f.spos.as<float4>();
    if (acc) TRY(upload4(acc_stage, acc, S.n, flags, f.st));
    TRY(f.clear_status());
    launch_validate_arrays(S.bpos(), vel ? S.bvel() : nullptr, (int)S.n, f.small(), f.nsm, f.st);
    f.launches += 1;
    // the one synchronisation: every caller buffer has been read once it returns
    TRY(f.read_small());
    if (f.h_small->status == ST_BAD_INPUT) {
        f.clear_status();
        return fail(BH_ERR_INVALID, "non-finite coordinate or non-positive mass");
    }
    // device-side copies only: later calls on the stream are ordered after them
    const size_t nb = (size_t)S.n * sizeof(float4);
    CKR(cudaMemcpyAsync(S.pos(), S.bpos(), nb, cudaMemcpyDeviceToDevice, f.st));
    if (vel) CKR(cudaMemcpyAsync(S.vel(), S.bvel(), nb, cudaMemcpyDeviceToDevice, f.st));
    if (acc) CKR(cudaMemcpyAsync(S.acc(), acc_stage, nb, cudaMemcpyDeviceToDevice, f.st));
    s->f.acc_valid = acc != nullptr;
    s->f.tree_valid = false;
    return BH_OK;
}

int bh_build_tree(bh_system *s)
{
    if (!s) return fail(BH_ERR_INVALID, "null system");
    TRY(s->f.begin_call());
    return s->f.build_only();
}

int bh_get_tree(bh_system *s, uint64_t *keys, uint32_t *order, bh_node *nodes, float *com_m,
                int64_t node_cap, int64_t *n_nodes, float *cube)
{
    if (!s) return fail(BH_ERR_INVALID, "null system");
    TRY(s->f.begin_call());
    return s->f.export_tree(0, keys, order, nodes, com_m, node_cap, n_nodes, cube);
}

int bh_compute_accel(bh_system *s, float *acc_out, unsigned flags)
{
    if (!s) return fail(BH_ERR_INVALID, "null system");
    TRY(s->f.begin_call());
    TRY(s->f.compute_accel());
    if (acc_out) {
        TRY(download4(acc_out, s->f.systems[0]->acc(), s->f.systems[0]->n, flags, s->f.st));
        TRY(s->f.sync());
    }
    return BH_OK;
}

int bh_step(bh_system *s, int nsteps, double dt, int use_graph)
{
    if (!s) return fail(BH_ERR_INVALID, "null system");
    if (nsteps < 0) return fail(BH_ERR_INVALID, "nsteps must be >= 0");
    if (!std::isfinite(dt)) return fail(BH_ERR_INVALID, "dt must be finite");
    TRY(s->f.begin_call());
    TRY(s->f.set_dt(dt));
    if (nsteps == 0) return s->f.acc_valid ? BH_OK : s->f.compute_accel();
    return s->f.step(nsteps, use_graph != 0);
}

int bh_get_state(bh_system *s, float *pos_mass, float *vel, float *acc, unsigned flags)
{
    if (!s) return fail(BH_ERR_INVALID, "null system");
    TRY(s->f.begin_call());
    SysState &S = *s->f.systems[0];
    if (pos_mass) TRY(download4(pos_mass, S.pos(), S.n, flags, s->f.st));
    if (vel) TRY(download4(vel, S.vel(), S.n, flags, s->f.st));
    if (acc) TRY(download4(acc, S.acc(), S.n, flags, s->f.st));
    return s->f.sync();
}

int bh_diagnostics(bh_system *s, double out[8])
{
    if (!s || !out) return fail(BH_ERR_INVALID, "null argument");
    TRY(s->f.begin_call());
    std::vector<double> v;
    TRY(s->f.diagnostics(v));
    std::memcpy(out, v.data(), 8 * sizeof(double));
    return BH_OK;
}

int bh_interaction_count(bh_system *s, uint32_t *counts, uint64_t *total)
{
    if (!s) return fail(BH_ERR_INVALID, "null system");
    TRY(s->f.begin_call());
    return s->f.interaction_count(0, counts, total);
}

int bh_walk_stats(bh_system *s, uint64_t *interactions, uint64_t *warp_iterations,
                  uint64_t *slot_visits)
{
    if (!s) return fail(BH_ERR_INVALID, "null system");
    TRY(s->f.begin_call());
    uint64_t tot = 0;
    TRY(s->f.interaction_count(0, nullptr, &tot));
    const Small &h = *s->f.h_small;
    if (interactions) *interactions = h.wstats[0];
    if (warp_iterations) *warp_iterations = h.wstats[1];
    if (slot_visits) *slot_visits = h.wstats[2];
    return BH_OK;
}

int bh_set_tuning(bh_system *s, const bh_tuning *t)
{
    if (!s) return fail(BH_ERR_INVALID, "null system");
    return s->f.set_tuning(t);
}

int bh_get_tuning(bh_system *s, bh_tuning *t)
{
    if (!s || !t) return fail(BH_ERR_INVALID, "null argument");
    *t = s->f.tune;
    return BH_OK;
}

int bh_autotune(bh_system *s, bh_tuning *best)
{
    if (!s) return fail(BH_ERR_INVALID, "null system");
    TRY(s->f.begin_call());
    return s->f.autotune(best);
}

int bh_profile_begin(bh_system *s)
{
    if (!s) return fail(BH_ERR_INVALID, "null system");
    s->f.profile_begin();
    return BH_OK;
}

int bh_profile_end(bh_system *s, double *phase_ms, int64_t *steps, int64_t *launches)
{
    if (!s) return fail(BH_ERR_INVALID, "null system");
    return s->f.profile_end(phase_ms, steps, launches);
}

// ---------------------------------------------------------------- forest

int bh_forest_create(bh_forest **out, int nsys, const bh_system_desc *d, void *stream,
                     unsigned flags)
{
    if (!out) return fail(BH_ERR_INVALID, "null out");
    *out = nullptr;
    if (nsys < 1 || !d) return fail(BH_ERR_INVALID, "need at least one system");
    if (flags & ~(BH_DEVICE_PTRS | BH_POTENTIAL | BH_NO_KAHAN | BH_OPEN_INSIDE | BH_QUADRUPOLE |
                  BH_OPEN_BMAX))
        return fail(BH_ERR_INVALID, "unknown flags");
    if ((flags & BH_QUADRUPOLE) && (flags & BH_NO_KAHAN))
        return fail(BH_ERR_INVALID, "BH_QUADRUPOLE needs Kahan sums");
    for (int s = 0; s < nsys; ++s) {
        if (d[s].n < 1 || !d[s].pos_mass) return fail(BH_ERR_INVALID, "system " + std::to_string(s) + ": n < 1 or null pos_mass");
        TRY(check_params(d[s].G, d[s].eps, d[s].theta));
    }
    std::unique_ptr<bh_forest> F(new (std::nothrow) bh_forest);
    if (!F) return fail(BH_ERR_OOM, "host allocation failed");
    Forest &f = F->f;
    TRY(f.init(stream, flags & (BH_POTENTIAL | BH_NO_KAHAN | BH_OPEN_INSIDE | BH_QUADRUPOLE |
                                BH_OPEN_BMAX)));
    f.tune.static_share = nsys > 1 ? 0 : f.tune.static_share;  // uneven tiles: all dynamic
    TRY(f.begin_call());
    for (int s = 0; s < nsys; ++s) {
        auto st = std::make_unique<SysState>();
        st->G = d[s].G; st->eps = d[s].eps; st->theta = d[s].theta; st->dt = d[s].dt;
        TRY(st->alloc(d[s].n));
        TRY(load_state(f, *st, d[s].pos_mass, d[s].vel, flags & BH_DEVICE_PTRS));
        f.systems.push_back(st.get());
        f.owned.push_back(std::move(st));
    }
    TRY(f.setup());
    if (flags & BH_DEVICE_PTRS) TRY(f.validate_device());
    TRY(f.sync());
    *out = F.release();
    return BH_OK;
}

int bh_forest_destroy(bh_forest *f)
{
    if (!f) return BH_OK;
    f->f.sync();
    delete f;
    return BH_OK;
}

int bh_forest_compute_accel(bh_forest *f)
{
    if (!f) return fail(BH_ERR_INVALID, "null forest");
    TRY(f->f.begin_call());
    return f->f.compute_accel();
}

int bh_forest_step(bh_forest *f, int nsteps, double dt, int use_graph)
{
    if (!f) return fail(BH_ERR_INVALID, "null forest");
    if (nsteps < 0) return fail(BH_ERR_INVALID, "nsteps must be >= 0");
    TRY(f->f.begin_call());
    if (dt > 0) TRY(f->f.set_dt(dt));
    if (nsteps == 0) return f->f.acc_valid ? BH_OK : f->f.compute_accel();
    return f->f.step(nsteps, use_graph != 0);
}

int bh_forest_get_state(bh_forest *f, int sys, float *pos_mass, float *vel, float *acc,
                        unsigned flags)
{
    if (!f) return fail(BH_ERR_INVALID, "null forest");
    if (sys < 0 || sys >= f->f.nsys) return fail(BH_ERR_INVALID, "system index out of range");
    TRY(f->f.begin_call());
    SysState &S = *f->f.systems[sys];
    if (pos_mass) TRY(download4(pos_mass, S.pos(), S.n, flags, f->f.st));
    if (vel) TRY(download4(vel, S.vel(), S.n, flags, f->f.st));
    if (acc) TRY(download4(acc, S.acc(), S.n, flags, f->f.st));
    return f->f.sync();
}

int bh_forest_set_tuning(bh_forest *f, const bh_tuning *t)
{
    if (!f) return fail(BH_ERR_INVALID, "null forest");
    return f->f.set_tuning(t);
}

int bh_forest_autotune(bh_forest *f, bh_tuning *best)
{
    if (!f) return fail(BH_ERR_INVALID, "null forest");
    TRY(f->f.begin_call());
    return f->f.autotune(best);
}

int bh_forest_info(bh_forest *f, int64_t *n_total, int64_t *n_nodes)
{
    if (!f) return fail(BH_ERR_INVALID, "null forest");
    if (n_total) *n_total = f->f.n_total;
    if (n_nodes) {
        TRY(f->f.read_small());
        *n_nodes = f->f.h_small->M;
    }
    return BH_OK;
}

int bh_forest_profile_begin(bh_forest *f)
{
    if (!f) return fail(BH_ERR_INVALID, "null forest");
    f->f.profile_begin();
    return BH_OK;
}

int bh_forest_profile_end(bh_forest *f, double *phase_ms, int64_t *steps, int64_t *launches)
{
    if (!f) return fail(BH_ERR_INVALID, "null forest");
    return f->f.profile_end(phase_ms, steps, launches);
}

// ---------------------------------------------------------- sharding

int bh_partition_systems(int nsys, const int64_t *n, int world, int *rank_of)
{
    if (nsys < 0 || world < 1) return fail(BH_ERR_INVALID, "nsys must be >= 0 and world >= 1");
    if (nsys > 0 && (!n || !rank_of)) return fail(BH_ERR_INVALID, "null sizes or output");
    std::vector<std::pair<double, int>> cost((size_t)nsys);
    for (int s = 0; s < nsys; ++s) {
        if (n[s] < 1) return fail(BH_ERR_INVALID, "system " + std::to_string(s) + ": size < 1");
        const double x = (double)n[s];
        cost[s] = {x * std::log2(std::max(x, 2.0)), s};
    }
    // longest first; equal costs in index order
    std::sort(cost.begin(), cost.end(), [](const std::pair<double, int> &a,
                                           const std::pair<double, int> &b) {
        return a.first != b.first ? a.first > b.first : a.second < b.second;
    });
    std::vector<double> load((size_t)world, 0.0);
    for (const auto &c : cost) {
        int r = 0;
        for (int q = 1; q < world; ++q)
            if (load[q] < load[r]) r = q;
        load[r] += c.first;
        rank_of[c.second] = r;
    }
    return BH_OK;
}

// ---------------------------------------------------------- micro-benchmarks

int bh_micro_fma_peak(double *gflops, void *stream)
{
    if (!gflops) return fail(BH_ERR_INVALID, "null out");
    *gflops = micro_fma_gflops((cudaStream_t)stream);
    CKR(cudaGetLastError());
    return *gflops > 0 ? BH_OK : fail(BH_ERR_CUDA, "fma micro-benchmark failed");
}

int bh_micro_l1_gather(double *gsectors, void *stream)
{
    if (!gsectors) return fail(BH_ERR_INVALID, "null out");
    *gsectors = micro_l1_sectors((cudaStream_t)stream);
    CKR(cudaGetLastError());
    return *gsectors > 0 ? BH_OK : fail(BH_ERR_OOM, "L1 micro-benchmark allocation failed");
}

int bh_micro_copy_bw(size_t bytes, double *gbs, void *stream)
{
    if (!gbs || bytes < 1024) return fail(BH_ERR_INVALID, "bad argument");
    *gbs = micro_copy_gbs(bytes, (cudaStream_t)stream);
    CKR(cudaGetLastError());
    return *gbs > 0 ? BH_OK : fail(BH_ERR_OOM, "copy micro-benchmark allocation failed");
}

}  // extern "C"

// ======================================================================
//                               server
// ======================================================================

namespace {

using Clock = std::chrono::steady_clock;

// First-fit sub-allocator over one region allocated up front (the server's
// device pool and its pinned staging buffer): taking and returning a region
// is host bookkeeping only, so the serving loop never calls an allocator.
struct Pool {
    static constexpr size_t kAlign = 256;
    char *base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_;  // offset -> length, disjoint, never adjacent

    static size_t round(size_t nb) { return (std::max<size_t>(nb, 1) + kAlign - 1) & ~(kAlign - 1); }
    void init(void *b, size_t nb)
    {
        base = static_cast<char *>(b);
        size = nb & ~(kAlign - 1);
        free_.clear();
        if (size) free_[0] = size;
    }
    void *take(size_t nb)
    {
        nb = round(nb);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < nb) continue;
            const size_t off = it->first, len = it->second;
            free_.erase(it);
            if (len > nb) free_[off + nb] = len - nb;
            return base + off;
        }
        return nullptr;
    }
    void give(void *p, size_t nb)
    {
        if (!p) return;
        nb = round(nb);
        size_t off = static_cast<size_t>(static_cast<char *>(p) - base);
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + nb == next->first) {  // merge with the following block
            nb += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {  // merge with the preceding block
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += nb;
                return;
            }
        }
        free_[off] = nb;
    }
};

struct Job {
    uint64_t ticket = 0;
    int64_t n = 0;
    double G = 1, eps = 0.01, theta = 0.5, dt = 1e-3;
    int nsteps = 0;
    std::vector<float> pm, vel;        // inputs, then outputs
    std::vector<float> acc;
    double submit_s = 0, admit_s = 0, done_s = 0;
    int steps_done = 0;
    int status = BH_OK;
    bool accel_done = false;
    size_t bytes = 0;
    std::unique_ptr<SysState> state;
    void *dev = nullptr;               // region of the device pool (state arrays)
    void *stage = nullptr;             // region of the pinned staging buffer
    size_t stage_bytes = 0;
    cudaEvent_t ev = nullptr;          // end of the job's upload, then of its download
};

// Device bytes a resident system needs: its state (five float4 arrays) plus
// its share of the forest's scratch (two key and two id buffers, the sorted
// copy, node counts and offsets) and of the node arrays (WNode 32 B, nodeR
// 16 B, nodeD 32 B, level-list entry 4 B; up to ~2 nodes per particle with
// the growth margin; in quadrupole mode also the second moments, under the
// b_max rule each cell's FP64 b_max^2).
size_t state_per_particle() { return 5 * 16; }
size_t scratch_per_particle(unsigned flags)
{
    return (8 + 8 + 4 + 4 + 16 + 4 + 4) + 2 * (32 + 16 + 32 + 4) +
           ((flags & BH_QUADRUPOLE) ? 2 * (6 * 8 + 2 * 16) : 0) +  // FP64 + FP32
           ((flags & BH_OPEN_BMAX) ? 2 * 8 : 0);
}
constexpr size_t kJobOverhead = 4096 * 64;
size_t job_bytes(int64_t n, unsigned flags)
{
    return (size_t)n * (state_per_particle() + scratch_per_particle(flags)) + kJobOverhead;
}

}  // namespace

// The server keeps, for its whole life, the device memory its budget allows:
// one pool of state arrays (sub-allocated per admitted request) and the
// forest's scratch sized for the most particles the budget can hold, plus a
// pinned host staging buffer.  Each tick runs one forest step over the
// resident systems without waiting for it; while it runs, the tick thread
// admits requests (takes pool regions, stages their particles and uploads
// them on a second stream) and delivers finished ones (their downloads,
// issued on that stream when their last step ended, overlap the next step).
// An admitted request joins the forest at the next tick, after its upload.
struct bh_server {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::unique_ptr<Job>> pending;
    std::vector<std::unique_ptr<Job>> resident;  // every job holding device memory
    std::map<uint64_t, std::unique_ptr<Job>> finished;
    std::map<uint64_t, int> where;  // 0 pending, 1 resident, 2 finished
    uint64_t next_ticket = 1;
    size_t budget = 0;
    int max_slots = 1;
    unsigned flags = 0;
    bool stop = false;
    size_t resident_bytes = 0;
    bh_server_stats stats{};
    Forest forest;
    cudaStream_t cp = nullptr;   // copies in and out
    DevBuf pool_mem;             // state arrays of resident systems
    Pool pool, staging;
    void *staging_mem = nullptr;  // pinned
    std::vector<cudaEvent_t> free_events;
    std::thread th;
    Clock::time_point t0;

    ~bh_server()
    {
        for (cudaEvent_t e : free_events) cudaEventDestroy(e);
        if (staging_mem) cudaFreeHost(staging_mem);
        if (cp) cudaStreamDestroy(cp);
    }

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

    cudaEvent_t take_event()
    {
        if (!free_events.empty()) {
            cudaEvent_t e = free_events.back();
            free_events.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return e;
    }

    // Device memory and staging of a job go back to the pools; bookkeeping
    // under mu is the caller's.
    void release(Job &j)
    {
        if (j.stage) staging.give(j.stage, j.stage_bytes);
        j.stage = nullptr;
        j.stage_bytes = 0;
        if (j.dev) pool.give(j.dev, SysState::bytes_for(j.n));
        j.dev = nullptr;
        j.state.reset();
        if (j.ev) free_events.push_back(j.ev);
        j.ev = nullptr;
    }

    int upload(Job &j);
    int download(Job &j);
    void admit(std::vector<Job *> &joining);
    void deliver(std::vector<Job *> &leaving, bool wait);
    void loop();
};

// Stages a job's particles in pinned memory and copies them to its pool
// region on the copy stream; j.ev marks the end of the copy.  A job larger
// than the whole staging buffer is copied from its own (pageable) arrays,
// which makes the host wait for that copy.
int bh_server::upload(Job &j)
{
    SysState &S = *j.state;
    const size_t nb = (size_t)j.n * sizeof(float4);
    const bool has_vel = !j.vel.empty();
    const float *src_pm = j.pm.data();
    const float *src_v = has_vel ? j.vel.data() : nullptr;
    if (j.stage) {
        char *p = static_cast<char *>(j.stage);
        std::memcpy(p, src_pm, nb);
        src_pm = reinterpret_cast<const float *>(p);
        if (has_vel) {
            std::memcpy(p + nb, src_v, nb);
            src_v = reinterpret_cast<const float *>(p + nb);
        }
    }
    CKR(cudaMemcpyAsync(S.pos(), src_pm, nb, cudaMemcpyHostToDevice, cp));
    if (has_vel) CKR(cudaMemcpyAsync(S.vel(), src_v, nb, cudaMemcpyHostToDevice, cp));
    else CKR(cudaMemsetAsync(S.vel(), 0, nb, cp));
    CKR(cudaMemsetAsync(S.acc(), 0, nb, cp));
    CKR(cudaEventRecord(j.ev, cp));
    return BH_OK;
}

// Copies a finished job's positions, velocities and accelerations out on the
// copy stream (into staging when it has room, else straight into the job's
// arrays, which makes the host wait); the forest's stream has finished the
// job's last step when this is called.
int bh_server::download(Job &j)
{
    SysState &S = *j.state;
    const size_t nb = (size_t)j.n * sizeof(float4);
    j.acc.resize((size_t)j.n * 4);
    j.vel.resize((size_t)j.n * 4);
    j.stage_bytes = 3 * nb;
    j.stage = staging.take(j.stage_bytes);
    float *dst[3] = {j.pm.data(), j.vel.data(), j.acc.data()};
    if (j.stage) {
        for (int k = 0; k < 3; ++k) dst[k] = reinterpret_cast<float *>(static_cast<char *>(j.stage) + k * nb);
    } else {
        j.stage_bytes = 0;
    }
    const float4 *src[3] = {S.pos(), S.vel(), S.acc()};
    for (int k = 0; k < 3; ++k) CKR(cudaMemcpyAsync(dst[k], src[k], nb, cudaMemcpyDeviceToHost, cp));
    CKR(cudaEventRecord(j.ev, cp));
    return BH_OK;
}

// FIFO admission: the head of the queue is admitted while a slot is free, the
// budget holds its bytes, and the pools have a region for its state (and for
// its staging, unless it is too large to stage at all).
void bh_server::admit(std::vector<Job *> &joining)
{
    for (;;) {
        Job *j = nullptr;
        {
            std::lock_guard<std::mutex> lk(mu);
            if (stop || pending.empty() || (int)resident.size() >= max_slots ||
                resident_bytes + pending.front()->bytes > budget)
                return;
            Job &h = *pending.front();
            void *dev = pool.take(SysState::bytes_for(h.n));
            if (!dev) return;
            const size_t in_bytes = (size_t)h.n * sizeof(float4) * (h.vel.empty() ? 1 : 2);
            void *stg = nullptr;
            if (in_bytes <= staging.size) {
                stg = staging.take(in_bytes);
                if (!stg) {
                    pool.give(dev, SysState::bytes_for(h.n));
                    return;
                }
            }
            std::unique_ptr<Job> u = std::move(pending.front());
            pending.pop_front();
            j = u.get();
            j->dev = dev;
            j->stage = stg;
            j->stage_bytes = stg ? in_bytes : 0;
            resident_bytes += j->bytes;
            j->admit_s = now();
            where[j->ticket] = 1;
            resident.push_back(std::move(u));
            stats.admitted++;
            stats.resident_systems = (int64_t)resident.size();
            stats.peak_resident_systems = std::max(stats.peak_resident_systems, stats.resident_systems);
            stats.resident_bytes = (int64_t)resident_bytes;
            stats.peak_resident_bytes = std::max(stats.peak_resident_bytes, stats.resident_bytes);
        }
        j->state = std::make_unique<SysState>();
        SysState &S = *j->state;
        S.G = j->G; S.eps = j->eps; S.theta = j->theta; S.dt = j->dt;
        S.place(j->n, j->dev);
        j->ev = take_event();
        int rc = j->ev ? upload(*j) : fail(BH_ERR_CUDA, "cudaEventCreate failed");
        if (rc != BH_OK) j->status = rc;
        joining.push_back(j);
    }
}

// Hands over the jobs whose downloads have finished (all of them, waiting,
// when `wait`): results into the job's own arrays, memory back to the pools.
void bh_server::deliver(std::vector<Job *> &leaving, bool wait)
{
    std::vector<Job *> ready;
    for (size_t k = 0; k < leaving.size();) {
        Job *j = leaving[k];
        bool done = true;
        if (j->ev) {
            const cudaError_t e = wait ? cudaEventSynchronize(j->ev) : cudaEventQuery(j->ev);
            if (e == cudaErrorNotReady) {
                done = false;
            } else if (e != cudaSuccess) {
                cudaGetLastError();
                if (j->status == BH_OK) j->status = fail(BH_ERR_CUDA, std::string("result copy: ") + cudaGetErrorString(e));
            }
        }
        if (!done) {
            ++k;
            continue;
        }
        if (j->status == BH_OK && j->stage) {
            const size_t nb = (size_t)j->n * sizeof(float4);
            const char *p = static_cast<const char *>(j->stage);
            std::memcpy(j->pm.data(), p, nb);
            std::memcpy(j->vel.data(), p + nb, nb);
            std::memcpy(j->acc.data(), p + 2 * nb, nb);
        }
        ready.push_back(j);
        leaving.erase(leaving.begin() + k);
    }
    if (ready.empty()) return;
    {
        std::lock_guard<std::mutex> lk(mu);
        for (Job *j : ready) {
            release(*j);
            for (size_t k = 0; k < resident.size(); ++k) {
                if (resident[k].get() != j) continue;
                std::unique_ptr<Job> u = std::move(resident[k]);
                resident.erase(resident.begin() + k);
                resident_bytes -= u->bytes;
                u->done_s = now();
                where[u->ticket] = 2;
                stats.completed++;
                finished[u->ticket] = std::move(u);
                break;
            }
        }
        stats.resident_systems = (int64_t)resident.size();
        stats.resident_bytes = (int64_t)resident_bytes;
    }
    cv_done.notify_all();
}

void bh_server::loop()
{
    cudaSetDevice(forest.dev);
    std::vector<Job *> run;      // systems of the forest (the step in flight, if any)
    std::vector<Job *> joining;  // uploads issued; they join at the next tick
    std::vector<Job *> leaving;  // downloads issued
    bool in_flight = false;
    bool dirty = true;
    for (;;) {
        // 1. host work while the step runs: deliver finished downloads, admit
        deliver(leaving, false);
        admit(joining);
        {
            std::unique_lock<std::mutex> lk(mu);
            if (stop) break;
            if (!in_flight && run.empty() && joining.empty()) {
                if (!leaving.empty()) {
                    lk.unlock();
                    deliver(leaving, true);
                    continue;
                }
                cv_work.wait(lk, [&] { return stop || !pending.empty(); });
                continue;
            }
        }
        // 2. finish the step in flight
        const double t_tick0 = now();
        if (in_flight) {
            int rc = forest.step_end();
            in_flight = false;
            int64_t ps = 0;
            for (Job *j : run) {
                if (rc != BH_OK) {
                    j->status = rc;
                    continue;
                }
                if (j->accel_done) {
                    j->steps_done++;
                    ps += j->n;
                }
                j->accel_done = true;
            }
            std::lock_guard<std::mutex> lk(mu);
            if (rc == BH_OK) {
                stats.ticks++;
                stats.particle_steps += ps;
            }
        }
        // 3. jobs that are done (or failed) leave; their downloads overlap the next step
        for (size_t k = 0; k < run.size();) {
            Job *j = run[k];
            if (j->status != BH_OK || j->steps_done >= j->nsteps) {
                if (j->status == BH_OK) {
                    const int rc = download(*j);
                    if (rc != BH_OK) j->status = rc;
                }
                leaving.push_back(j);
                run.erase(run.begin() + k);
                dirty = true;
            } else {
                ++k;
            }
        }
        // 4. admitted jobs join (their uploads were issued a tick ago)
        for (Job *j : joining) {
            if (j->status == BH_OK && j->ev) {
                const cudaError_t e = cudaEventSynchronize(j->ev);
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    j->status = fail(BH_ERR_CUDA, std::string("request upload: ") + cudaGetErrorString(e));
                }
            }
            if (j->stage) {
                std::lock_guard<std::mutex> lk(mu);
                staging.give(j->stage, j->stage_bytes);
                j->stage = nullptr;
                j->stage_bytes = 0;
            }
            if (j->status == BH_OK) {
                run.push_back(j);
                dirty = true;
            } else {
                leaving.push_back(j);
            }
        }
        joining.clear();
        // 5. launch the next step over the resident systems
        if (!run.empty()) {
            int rc = BH_OK;
            if (dirty) {
                forest.systems.clear();
                for (Job *j : run) forest.systems.push_back(j->state.get());
                rc = forest.setup();
                dirty = false;
            }
            if (rc == BH_OK) {
                std::vector<int> modes(run.size());
                for (size_t k = 0; k < run.size(); ++k) modes[k] = run[k]->accel_done ? MODE_KDK : MODE_ACCEL;
                rc = forest.set_modes(modes);
            }
            if (rc == BH_OK) rc = forest.step_begin();
            if (rc == BH_OK) {
                in_flight = true;
            } else {
                for (Job *j : run) {
                    j->status = rc;
                    leaving.push_back(j);
                }
                run.clear();
                dirty = true;
            }
        }
        std::lock_guard<std::mutex> lk(mu);
        stats.busy_s += now() - t_tick0;
    }
    // shutdown: let the device finish, then cancel everything
    if (in_flight) forest.step_end();
    forest.sync();
    cudaStreamSynchronize(cp);
    std::lock_guard<std::mutex> lk(mu);
    for (auto &j : pending) {
        j->status = BH_ERR_CANCELLED;
        where[j->ticket] = 2;
        finished[j->ticket] = std::move(j);
    }
    pending.clear();
    for (auto &j : resident) {
        j->status = BH_ERR_CANCELLED;
        release(*j);
        where[j->ticket] = 2;
        finished[j->ticket] = std::move(j);
    }
    resident.clear();
    resident_bytes = 0;
    cv_done.notify_all();
}

extern "C" {

int bh_server_create(bh_server **out, size_t hbm_budget, int max_slots, void *stream,
                     unsigned flags)
{
    if (!out) return fail(BH_ERR_INVALID, "null out");
    *out = nullptr;
    if (max_slots < 1 || hbm_budget < (1u << 20)) return fail(BH_ERR_INVALID, "bad budget or slot count");
    if (flags & ~(BH_POTENTIAL | BH_NO_KAHAN | BH_OPEN_INSIDE | BH_QUADRUPOLE | BH_OPEN_BMAX))
        return fail(BH_ERR_INVALID, "unknown flags");
    if ((flags & BH_QUADRUPOLE) && (flags & BH_NO_KAHAN))
        return fail(BH_ERR_INVALID, "BH_QUADRUPOLE needs Kahan sums");
    std::unique_ptr<bh_server> s(new (std::nothrow) bh_server);
    if (!s) return fail(BH_ERR_OOM, "host allocation failed");
    s->budget = hbm_budget;
    s->max_slots = max_slots;
    s->flags = flags;
    TRY(s->forest.init(stream, flags));
    s->forest.adaptive_deep = false;
    // requests differ widely in cost per tile: all tiles in per-SM ranges,
    // balanced by taking from neighbouring ranges (served 3.45e8 particle-
    // steps/s against 3.20e8 with every tile from the global queue)
    s->forest.tune.static_share = 100;
    // the budget, carved once: the most particles it can hold resident, their
    // state arrays in one pool and the forest's scratch sized for them
    const size_t per = state_per_particle() + scratch_per_particle(flags);
    const int64_t n_max = (int64_t)std::min<size_t>(hbm_budget / per, (size_t)1 << 30);
    if (n_max < 1) return fail(BH_ERR_INVALID, "budget holds no particle");
    const size_t pool_bytes = SysState::bytes_for(n_max) + (size_t)max_slots * Pool::kAlign;
    TRY(s->pool_mem.ensure(pool_bytes));
    s->pool.init(s->pool_mem.p, pool_bytes);
    TRY(s->forest.reserve(n_max, std::min<int64_t>(max_slots, n_max)));
    // pinned staging: a slice of the budget, between 64 MiB and 1 GiB
    const size_t stage_bytes = std::min<size_t>(std::max<size_t>(hbm_budget / 64, 64u << 20), 1u << 30);
    if (cudaMallocHost(&s->staging_mem, stage_bytes) != cudaSuccess) {
        cudaGetLastError();
        s->staging_mem = nullptr;
        return fail(BH_ERR_OOM, "pinned staging allocation failed");
    }
    s->staging.init(s->staging_mem, stage_bytes);
    CKR(cudaStreamCreateWithFlags(&s->cp, cudaStreamNonBlocking));
    CKR(cudaStreamSynchronize(s->forest.st));
    s->t0 = Clock::now();
    bh_server *raw = s.get();
    try {
        s->th = std::thread([raw] { raw->loop(); });
    } catch (...) {
        return fail(BH_ERR_OOM, "could not start the server thread");
    }
    *out = s.release();
    return BH_OK;
}

int bh_submit(bh_server *s, const bh_request *r, uint64_t *ticket)
{
    if (!s || !r || !ticket) return fail(BH_ERR_INVALID, "null argument");
    if (r->n < 1 || r->n > (1ll << 30) || !r->pos_mass) return fail(BH_ERR_INVALID, "bad request size or null pos_mass");
    if (r->nsteps < 0) return fail(BH_ERR_INVALID, "nsteps must be >= 0");
    if (!std::isfinite(r->dt)) return fail(BH_ERR_INVALID, "dt must be finite");
    TRY(check_params(r->G, r->eps, r->theta));
    if (!finite_state(r->n, r->pos_mass, r->vel)) return fail(BH_ERR_INVALID, "non-finite coordinate or non-positive mass");
    auto j = std::make_unique<Job>();
    j->n = r->n;
    j->G = r->G; j->eps = r->eps; j->theta = r->theta; j->dt = r->dt;
    j->nsteps = r->nsteps;
    j->bytes = job_bytes(r->n, s->flags);
    if (j->bytes > s->budget) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stats.rejected++;
        return fail(BH_ERR_BUDGET, "request needs " + std::to_string(j->bytes) + " bytes, budget is " + std::to_string(s->budget));
    }
    j->pm.assign(r->pos_mass, r->pos_mass + 4 * r->n);
    if (r->vel) j->vel.assign(r->vel, r->vel + 4 * r->n);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return fail(BH_ERR_CANCELLED, "server is shutting down");
    j->ticket = s->next_ticket++;
    j->submit_s = s->now();
    *ticket = j->ticket;
    s->where[j->ticket] = 0;
    s->pending.push_back(std::move(j));
    s->stats.submitted++;
    s->cv_work.notify_one();
    return BH_OK;
}

static int take_result(bh_server *s, uint64_t ticket, bh_result *res)
{
    // caller holds s->mu
    auto it = s->finished.find(ticket);
    Job &j = *it->second;
    if (res) {
        res->status = j.status;
        res->submit_s = j.submit_s;
        res->admit_s = j.admit_s;
        res->done_s = j.done_s;
        res->steps_done = j.steps_done;
        if (j.status == BH_OK) {
            const size_t nb = sizeof(float) * 4 * (size_t)j.n;
            if (res->pos_mass) std::memcpy(res->pos_mass, j.pm.data(), nb);
            if (res->vel) std::memcpy(res->vel, j.vel.data(), nb);
            if (res->acc) std::memcpy(res->acc, j.acc.data(), nb);
        }
    }
    const int st = j.status;
    s->finished.erase(it);
    s->where.erase(ticket);
    if (st != BH_OK) return fail(st, "request failed with status " + std::to_string(st));
    return BH_OK;
}

int bh_poll(bh_server *s, uint64_t ticket, bh_result *res)
{
    if (!s) return fail(BH_ERR_INVALID, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto w = s->where.find(ticket);
    if (w == s->where.end()) return fail(BH_ERR_INVALID, "unknown ticket");
    if (w->second != 2) return BH_PENDING;
    return take_result(s, ticket, res);
}

int bh_wait(bh_server *s, uint64_t ticket, bh_result *res, double timeout_s)
{
    if (!s) return fail(BH_ERR_INVALID, "null server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto w = s->where.find(ticket);
    if (w == s->where.end()) return fail(BH_ERR_INVALID, "unknown ticket");
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(std::max(0.0, timeout_s)));
    while (s->where[ticket] != 2) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && s->where[ticket] != 2)
            return fail(BH_ERR_TIMEOUT, "request not finished within the timeout");
    }
    return take_result(s, ticket, res);
}

int bh_server_stats_get(bh_server *s, bh_server_stats *st)
{
    if (!s || !st) return fail(BH_ERR_INVALID, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *st = s->stats;
    return BH_OK;
}

double bh_server_now(bh_server *s) { return s ? s->now() : 0.0; }

int bh_server_destroy(bh_server *s)
{
    if (!s) return BH_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->th.joinable()) s->th.join();
    s->forest.sync();
    delete s;
    return BH_OK;
}

}  // extern "C"

namespace bh {
// Lets other translation units report through bh_last_error().
void set_last_error(const std::string &msg) { g_err = msg; }
}  // namespace bh
