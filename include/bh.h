/*
 * bh.h -- C ABI of the GB300 Barnes-Hut library (libbh.so).
 *
 * The library computes the data-parallel hot path of the Barnes-Hut method as
 * studied in Dekate et al., "Improving the scalability of parallel N-body
 * applications with an event driven constraint based execution model"
 * (arXiv:1109.5190):
 *   - Section I: n particles evolve under pairwise gravitational forces; the
 *     particles are grouped in a hierarchy of cubes subdivided until each
 *     holds one particle, and a centre of mass is kept per cube.
 *   - Section III, Fig. 1: a remote cluster is replaced by a single body when
 *     it is far enough away relative to its size, theta setting the error.
 *   - Section III: a global barrier at tree construction in every iteration,
 *     then the force computation, the most expensive stage.
 * What the paper leaves unstated is fixed as follows (the same readings as
 * the test oracle): Plummer-softened Newtonian forces; the opening test
 * s^2 < theta^2 d^2 with s = side / 2^level and d the distance to the cell's
 * centre of mass, leaves taken particle by particle; 63-bit Morton keys from a
 * 21-bit FP32 quantisation of the bounding cube; a depth cap of 21 levels,
 * where coincident points share one leaf; kick-drift-kick leapfrog.
 *
 * Conventions for every call:
 *   - Return value: BH_OK (0) on success, BH_PENDING (1) from bh_poll when a
 *     result is not ready, a negative BH_ERR_* code otherwise.  Nothing traps
 *     on the device; device-side failures (node capacity, bounded waits) come
 *     back as status codes.  bh_last_error() returns a message for the last
 *     failing call on the calling thread.
 *   - Particle arrays are float32, 4 values per particle: pos_mass = (x, y, z,
 *     m), vel = (vx, vy, vz, unused), acc = (ax, ay, az, phi).  They are in
 *     the caller's particle order (particle i is row i) for input and output.
 *   - Pointers are host pointers unless the call's flags include
 *     BH_DEVICE_PTRS, in which case they are device pointers readable or
 *     writable on the system's stream during the call only.  The caller keeps
 *     ownership of every array it passes; the library copies what it keeps.
 *   - Every call that returns BH_OK has finished its device work (the stream
 *     is synchronised) unless its comment says otherwise.
 *   - Handles are not thread-safe: one thread at a time per handle.  A
 *     bh_server handle may be used from any thread.
 */
#ifndef BH_H
#define BH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define BH_OK             0
#define BH_PENDING        1
#define BH_ERR_INVALID   (-1)  /* bad argument (size, pointer, parameter value) */
#define BH_ERR_OOM       (-2)  /* device or host allocation failed */
#define BH_ERR_BUDGET    (-3)  /* request larger than the server's HBM budget */
#define BH_ERR_CAPACITY  (-4)  /* node buffer overflow that could not be recovered */
#define BH_ERR_TIMEOUT   (-5)  /* a bounded wait expired */
#define BH_ERR_CUDA      (-6)  /* a CUDA runtime call failed */
#define BH_ERR_STATE     (-7)  /* call not valid in the handle's current state */
#define BH_ERR_CANCELLED (-8)  /* request cancelled or server shut down */

/* ------------------------------------------------------------------- flags */
#define BH_DEVICE_PTRS  0x1u  /* pointer arguments are device pointers */
#define BH_POTENTIAL    0x2u  /* the walk also accumulates phi (needed for PE) */
#define BH_NO_KAHAN     0x4u  /* plain FP32 force sums instead of Kahan sums */
#define BH_OPEN_INSIDE  0x8u  /* alternative opening rule: a cell that contains
                                 the particle is always opened (the pure test of
                                 Section III can accept it for theta > 1/sqrt(3));
                                 the walk then runs one particle per lane */
#define BH_QUADRUPOLE   0x10u /* accepted cells add their quadrupole term
                                 (second moments about the centre of mass,
                                 softened kernel expanded to second order);
                                 one particle per lane, Kahan sums required */
#define BH_OPEN_BMAX    0x20u /* alternative size in the opening test
                                 (Section V: other ways of computing the
                                 criterion): a cell is accepted iff
                                 b_max^2 < theta^2 d^2, b_max = distance from
                                 its centre of mass to the farthest corner of
                                 its cube, instead of s^2 < theta^2 d^2; for
                                 theta <= 1 a cell holding the particle is then
                                 never accepted.  The split walk (group 0) is
                                 not available under it (a group-0 tuning runs
                                 as group 1) */

#define BH_MAX_DEPTH 21       /* levels below the root; fixed by the key width */

/* Solver parameters of one system.
 *   G      gravitational constant (> 0)
 *   eps    Plummer softening length (>= 0; 0 allowed, coincident pairs are
 *          then skipped)
 *   theta  opening parameter (>= 0; 0 = direct summation through the tree)
 *   max_depth must be BH_MAX_DEPTH, leaf_cap must be 1 (one particle per
 *          leaf, Section I; only coincident points share a leaf)
 *   flags  BH_POTENTIAL, BH_NO_KAHAN */
typedef struct bh_params {
    double G, eps, theta;
    int max_depth;
    int leaf_cap;
    unsigned flags;
} bh_params;

/* One node of the exported canonical tree: depth-first pre-order, children
 * in octant order 4x+2y+z, which is Morton order of (level, prefix).
 *   prefix    the node's top 3*level key bits
 *   first     index of its first particle in sorted (key, input index) order
 *   count     particles in the node
 *   level     0 = root ... 21
 *   childmask bit o set when the child in octant o exists (0 for leaves) */
typedef struct bh_node {
    uint64_t prefix;
    uint32_t first;
    uint32_t count;
    uint8_t level;
    uint8_t childmask;
    uint8_t pad[6];
} bh_node;

/* Walk launch shape (the autotuner's search space).
 *   ppl             particles per lane (1, 2 or 4; 4 only with group 1 or 32):
 *                   a warp task is a tile of 32*ppl consecutive Morton-sorted
 *                   particles; with group < 32 a lane's particles are
 *                   neighbours in that order
 *   warps_per_block 1..16
 *   blocks_per_sm   0 = as many as fit
 *   group           lanes that vote together on the next node (1, 2, 4, 8 or
 *                   32): 32 = the warp walks the union of its particles'
 *                   traversals (one broadcast node load per step), 4 or 8 =
 *                   aligned lane groups each walk their own union, 1 = every
 *                   lane walks its own particles' traversal.  0 = split walk
 *                   (ppl 1): the warp walks the union of the top levels
 *                   (level <= clamp(floor(log8 n) - 3, 2, 5)), then every lane
 *                   walks the subtrees below them that it opened on its own.
 *                   BH_GROUP_LIST (64) = interaction lists (ppl 1): the warp
 *                   walks the union of its tile's traversals into a list of
 *                   (node, lanes that take it), then evaluates the list.
 *                   BH_GROUP_SIBLINGS (65) = one lane per particle (ppl 1,
 *                   no vote) over a copy of the node records built after each
 *                   tree in which every node's children sit next to each
 *                   other, so lanes at sibling nodes share cache lines.  Not
 *                   available with BH_OPEN_INSIDE, BH_QUADRUPOLE or
 *                   BH_OPEN_BMAX (it runs as group 1 there).  Measured
 *                   slower than group 1 on the workloads tried, so
 *                   bh_autotune does not consider it (nor BH_GROUP_LIST).
 * Accelerations are bit-identical for every shape with group >= 1 (the
 * interaction lists and the sibling-order walk included).  The split
 * walk sums the same terms in another order, fixed by each particle's tile (32
 * consecutive sorted particles of its system), so its results are
 * bit-identical among split shapes, alone or in a forest, and differ from the
 * others only by rounding; interaction counts are the same for every shape. */
#define BH_GROUP_LIST 64
#define BH_GROUP_SIBLINGS 65

typedef struct bh_tuning {
    int ppl;
    int warps_per_block;
    int blocks_per_sm;
    int group;
    int static_share;  /* percent (0..100) of the tiles split into one
                          contiguous range per SM, which the SM's blocks share
                          (neighbouring walks share L1); an SM whose range is
                          empty takes tiles from the back of its neighbours'
                          ranges; the rest are handed out by an atomic queue */
} bh_tuning;

typedef struct bh_system bh_system;
typedef struct bh_forest bh_forest;
typedef struct bh_server bh_server;

/* Message for the last failing call on this thread ("" if none). */
const char *bh_last_error(void);

/* Library version string. */
const char *bh_version(void);

/* Fills *p with G = 1, eps = 0.01, theta = 0.5, max_depth = 21, leaf_cap = 1,
 * flags = 0. */
int bh_params_default(bh_params *p);

/* ---------------------------------------------------------- single system */

/* Creates a system of n >= 1 particles and copies its state to the device.
 * pos_mass: n x 4 (x, y, z, m), masses > 0 and coordinates finite (checked;
 * BH_ERR_INVALID otherwise).  vel: n x 4 or NULL (zero velocities).
 * stream: a cudaStream_t to run on, or NULL for a stream the library creates.
 * flags: BH_DEVICE_PTRS when pos_mass / vel are device pointers.
 * The library owns the device state until bh_destroy. */
int bh_create(bh_system **out, const bh_params *p, int64_t n, const float *pos_mass,
              const float *vel, void *stream, unsigned flags);

int bh_destroy(bh_system *s);

/* Replaces the state (n x 4 each).  vel NULL keeps the current velocities.
 * acc, if not NULL, is taken as the acceleration of the new positions (as
 * returned by bh_get_state), so the next bh_step needs no extra force
 * evaluation; if NULL the stored acceleration is invalidated.  The new state
 * is checked on the device first (finite coordinates and velocities,
 * positive masses): BH_ERR_INVALID leaves the old state in place.  On return
 * the caller's buffers have been read and may be reused. */
int bh_set_state(bh_system *s, const float *pos_mass, const float *vel, const float *acc,
                 unsigned flags);

/* Builds the octree of the current positions (Section I; the tree-build
 * barrier of Section III): bounding cube and root centre of mass (FP64),
 * Morton keys, radix sort by (key, input index), canonical topology with the
 * depth cap, bottom-up masses and centres of mass (FP64, kept for the walk
 * as an FP32 value plus its FP32-rounded remainder). */
int bh_build_tree(bh_system *s);

/* Copies the last built tree to host memory (for parity checks).
 * keys: n sorted keys or NULL; order: n input indices in sorted order or NULL;
 * nodes: node_cap entries or NULL; com_m: node_cap x 4 floats (centre of
 * mass, mass) or NULL.  *n_nodes receives the node count; BH_ERR_INVALID if it
 * exceeds node_cap while nodes or com_m is given.  cube (4 floats: lo_x,
 * lo_y, lo_z, side) may be NULL. */
int bh_get_tree(bh_system *s, uint64_t *keys, uint32_t *order, bh_node *nodes,
                float *com_m, int64_t node_cap, int64_t *n_nodes, float *cube);

/* Builds the tree and walks it (Section III: the force computation):
 * a_i = G sum over accepted cells and leaf particles of
 * m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^(3/2), per particle exactly as the
 * opening test decides for that particle.  The result is kept as the
 * system's acceleration; if acc_out is not NULL it also receives n x 4 floats
 * (ax, ay, az, phi; phi is 0 unless BH_POTENTIAL). */
int bh_compute_accel(bh_system *s, float *acc_out, unsigned flags);

/* Advances nsteps kick-drift-kick leapfrog steps of size dt, rebuilding the
 * tree every step.  Computes the initial acceleration first if the system has
 * none.  use_graph != 0 captures the step loop in a CUDA graph (cached per
 * nsteps and dt).  A node-buffer overflow inside a step is detected on the
 * device, the step is rolled back, the buffer grown and the step redone. */
int bh_step(bh_system *s, int nsteps, double dt, int use_graph);

/* Copies the state out (each pointer may be NULL). */
int bh_get_state(bh_system *s, float *pos_mass, float *vel, float *acc, unsigned flags);

/* FP64 conserved quantities out[8] = {KE, PE, Px, Py, Pz, COMx, COMy, COMz}.
 * PE needs phi from the last walk (BH_POTENTIAL); it is NaN otherwise. */
int bh_diagnostics(bh_system *s, double out[8]);

/* Walks the current tree once more counting, per particle, the accepted
 * cells plus leaf particles it interacts with (its own leaf included).
 * counts: n uint32 in input order or NULL; *total receives the sum. */
int bh_interaction_count(bh_system *s, uint32_t *counts, uint64_t *total);

/* Work of one walk over the current tree (the counting walk above):
 * interactions (accepted cells + leaf particles, summed over particles), warp
 * iterations (nodes the warps visit: the union of their particles' walks) and
 * particle-slot visits (nodes each particle itself visits, opened or taken).
 * interactions / (32 x warp_iterations) is the walk's lane efficiency. */
int bh_walk_stats(bh_system *s, uint64_t *interactions, uint64_t *warp_iterations,
                  uint64_t *slot_visits);

/* Walk launch shape: set explicitly, or pick by timing the candidates on the
 * current tree (cached per device, log2 N bucket and theta bucket).  Results
 * do not depend on the shape. */
int bh_set_tuning(bh_system *s, const bh_tuning *t);
int bh_get_tuning(bh_system *s, bh_tuning *t);
int bh_autotune(bh_system *s, bh_tuning *best);

/* ------------------------------------------------------------- profiling */

#define BH_NPHASE 3  /* 0 integrate (kicks, drift), 1 tree build, 2 walk */

/* Starts recording CUDA events around the phases of each step on the
 * system's stream. */
int bh_profile_begin(bh_system *s);
/* Stops recording; phase_ms[BH_NPHASE] receives the summed device time of
 * each phase, *steps the steps recorded, *launches the kernels launched. */
int bh_profile_end(bh_system *s, double *phase_ms, int64_t *steps, int64_t *launches);

/* ------------------------------------------------------------------ forest */

/* One system of a forest.  dt is the step size used when bh_forest_step is
 * given dt <= 0. */
typedef struct bh_system_desc {
    int64_t n;
    const float *pos_mass;  /* n x 4 */
    const float *vel;       /* n x 4 or NULL */
    double G, eps, theta, dt;
} bh_system_desc;

/* Many independent systems sharing one set of launches per step: a segmented
 * sort, one topology / centre-of-mass pass and one persistent walk launch
 * over all trees.  Each system's tree and accelerations are the same as it
 * would get alone.  flags: BH_DEVICE_PTRS, BH_POTENTIAL, BH_NO_KAHAN. */
int bh_forest_create(bh_forest **out, int nsys, const bh_system_desc *d, void *stream,
                     unsigned flags);
int bh_forest_destroy(bh_forest *f);
int bh_forest_compute_accel(bh_forest *f);
/* nsteps KDK steps for every system (dt > 0 overrides each system's dt);
 * use_graph != 0 captures the nsteps loop in one CUDA graph. */
int bh_forest_step(bh_forest *f, int nsteps, double dt, int use_graph);
int bh_forest_get_state(bh_forest *f, int sys, float *pos_mass, float *vel, float *acc,
                        unsigned flags);
int bh_forest_set_tuning(bh_forest *f, const bh_tuning *t);
int bh_forest_autotune(bh_forest *f, bh_tuning *best);
/* Total particles and node count of the last build. */
int bh_forest_info(bh_forest *f, int64_t *n_total, int64_t *n_nodes);
/* Phase timing of the forest's steps, as bh_profile_begin / bh_profile_end:
 * phase_ms[BH_NPHASE] sums the device time of each phase over all systems. */
int bh_forest_profile_begin(bh_forest *f);
int bh_forest_profile_end(bh_forest *f, double *phase_ms, int64_t *steps, int64_t *launches);

/* Deals nsys independent systems of sizes n[0..nsys) to `world` ranks (one
 * GPU each) for a run sharded by system: rank_of[s] receives the rank of
 * system s.  The paper's conclusion (Section VI) names distributed runs as the
 * next step; systems of a forest or a request stream are independent, so a
 * rank needs nothing from another but the final gather of results.  The cost
 * of a system is taken as n log2 n (the walk's work at a fixed theta); systems
 * are assigned longest first, each to the rank with the least cost so far
 * (ties: the lower system index first, the lower rank), which keeps the
 * largest rank cost within 4/3 of the best possible.  Deterministic: every
 * rank calling it with the same sizes gets the same assignment.  Host only
 * (no device work).  BH_ERR_INVALID for nsys < 0, world < 1, a size < 1 or
 * null arrays with nsys > 0. */
int bh_partition_systems(int nsys, const int64_t *n, int world, int *rank_of);

/* ------------------------------------------------------------------ server */

/* A solve request: particles (host arrays, copied at submit), parameters,
 * step count (0 = one force evaluation only) and step size. */
typedef struct bh_request {
    int64_t n;
    const float *pos_mass;  /* n x 4, host */
    const float *vel;       /* n x 4 or NULL, host */
    double G, eps, theta, dt;
    int nsteps;
    unsigned flags;         /* BH_POTENTIAL, BH_NO_KAHAN */
} bh_request;

/* Result of a finished request.  Output arrays are supplied by the caller
 * (host, n x 4 each, may be NULL) and filled by bh_poll. */
typedef struct bh_result {
    int status;             /* BH_OK or the request's error */
    int pad;
    float *pos_mass;
    float *vel;
    float *acc;
    double submit_s;        /* times on the server's monotonic clock */
    double admit_s;
    double done_s;
    int64_t steps_done;
} bh_result;

typedef struct bh_server_stats {
    int64_t submitted, admitted, completed, rejected;
    int64_t ticks;                /* forest steps run */
    int64_t particle_steps;       /* sum over ticks of resident particles stepped */
    int64_t resident_systems;
    int64_t peak_resident_systems;
    int64_t resident_bytes, peak_resident_bytes;
    double busy_s;                /* time spent running ticks */
} bh_server_stats;

/* Starts a server thread that admits requests while their device memory
 * fits hbm_budget bytes and a slot is free (max_slots), keeps admitted
 * systems resident on the device, and runs one forest step per tick over
 * every resident system: a request arriving while others run joins the
 * batch at the next tick (continuous batching).  stream may be NULL. */
int bh_server_create(bh_server **out, size_t hbm_budget, int max_slots, void *stream,
                     unsigned flags);
/* Queues a request; *ticket identifies it.  BH_ERR_BUDGET if the request
 * alone exceeds the budget. */
int bh_submit(bh_server *s, const bh_request *r, uint64_t *ticket);
/* BH_PENDING while the request runs; BH_OK once done, with res filled and
 * the ticket released.  Returns the request's own error if it failed. */
int bh_poll(bh_server *s, uint64_t ticket, bh_result *res);
/* Waits up to timeout_s seconds for the ticket (BH_ERR_TIMEOUT if it does
 * not finish), then behaves like bh_poll. */
int bh_wait(bh_server *s, uint64_t ticket, bh_result *res, double timeout_s);
int bh_server_stats_get(bh_server *s, bh_server_stats *st);
/* Seconds on the server's monotonic clock (the clock of bh_result times). */
double bh_server_now(bh_server *s);
/* Stops the thread; pending and running requests end with BH_ERR_CANCELLED. */
int bh_server_destroy(bh_server *s);

/* ------------------------------------------------- allocation-free Morton keys */

/* The paper has no counterpart to this call: it exists for callers that
 * cannot allocate device memory.  cudaMalloc may wait until the whole device
 * is idle and fails when another allocator (a framework's caching allocator,
 * a pre-carved pool) already holds the free memory; code on a latency-critical
 * loop, or code that owns no allocator, can still compute keys here.
 *
 * Computes, for n particles (pos_mass: device, n x 4 floats), the same 63-bit
 * Morton keys as the tree build (keys: device, n uint64, input order) and the
 * key cube (cube: device, 4 floats lo_x, lo_y, lo_z, side; may be NULL).
 * Masses are not read.  Each pointer must be memory of the current device (or
 * managed memory), pos_mass 16-byte, keys 8-byte and cube 4-byte aligned;
 * anything else (a host pointer, another device's memory, an offset that
 * breaks the alignment) returns BH_ERR_INVALID before any work is enqueued.
 * Allocates nothing and calls no allocating routine: its only scratch is a
 * file-scope device array of 128 KiB + 32 bytes (per-chunk boxes), held on
 * every GPU that loads the library until the process exits.  n must be in
 * [1, BH_NOALLOC_MAX_N]; larger n returns BH_ERR_INVALID with a message.
 * The work is enqueued on `stream` (NULL = legacy default stream) and the call
 * returns without synchronising, so input the tree build would reject cannot
 * come back as a status: if any coordinate is non-finite, every key is set to
 * BH_NOALLOC_BAD_KEY (no 63-bit key has that value) and the cube to NaN.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the rest
 * of the process; make that first call before any stream capture.  A
 * cudaDeviceReset ends the context holding the array, so the kept address is
 * stale afterwards: do not call this entry point again in that process (the
 * library's other handles do not survive a reset either).  Every call on a
 * device shares its array and overwrites what it reads, so calls whose work
 * overlaps on one GPU race: keep them on one stream or order them. */
#define BH_NOALLOC_MAX_N 16777216
#define BH_NOALLOC_BAD_KEY 0xffffffffffffffffull
int bh_morton_keys_noalloc(const float *pos_mass, int64_t n, uint64_t *keys, float *cube,
                           void *stream);

/* ---------------------------------------------------------- micro-benchmarks */

/* Measured FP32 non-tensor throughput: a kernel of independent FMA chains on
 * every SM; *gflops = 2 x FMAs / time. */
int bh_micro_fma_peak(double *gflops, void *stream);
/* Measured L1 throughput of the walk's kind of load: every lane reads its
 * own pseudo-random 32-byte record (one 256-bit load) from a table that stays
 * in L1, 48 warps per SM.  *gsectors = distinct 32-byte sectors delivered per
 * second (in units of 1e9), the ceiling for a walk in which each lane sits at
 * its own node. */
int bh_micro_l1_gather(double *gsectors, void *stream);
/* Measured device copy bandwidth over a buffer of `bytes` (read + write
 * counted). */
int bh_micro_copy_bw(size_t bytes, double *gbs, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* BH_H */
