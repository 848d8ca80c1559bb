/*
 * bh_oracle.c -- plain, slow, FP64 CPU oracle for the Barnes-Hut hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load or run this file.  The GPU library neither links nor
 * calls it, and it shares no code, header or table with the GPU library.
 *
 * What it computes follows the paper (Dekate et al., arXiv:1109.5190):
 *   - Section I: the N-body problem -- n particles evolving under pairwise
 *     gravity -- and the Barnes-Hut octree, whose cubes are split into eight
 *     until each leaf holds a single particle, with a centre of mass per cube.
 *   - Section III (Fig. 1): a remote cluster is replaced by one body when the
 *     distance D to it exceeds r/theta; smaller theta means smaller error.
 *   - Section III (Fig. 2): a worked 2-D example where a cluster of two
 *     particles is replaced by its centroid, so the two remote particles each
 *     need only two inputs.
 * The paper states neither the force law, nor the integrator, nor the key
 * construction; the readings used here are:
 *   - force: Plummer-softened Newtonian gravity,
 *       a_i = G sum_j m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^(3/2);
 *     a term whose softened squared distance is exactly 0 contributes nothing
 *     (this removes the self term when eps = 0);
 *   - potential: phi_i = -G sum_{j != i} m_j / sqrt(|x_j - x_i|^2 + eps^2) for
 *     particles reached individually, -G M / sqrt(d^2 + eps^2) for an accepted
 *     cell (its total mass M at distance d to its centre of mass);
 *   - opening test: a cell of side s = side / 2^level at distance d from the
 *     particle (d measured to the cell's centre of mass) is accepted as one
 *     body iff s^2 < theta^2 d^2 (strict); theta = 0 never accepts, which is
 *     direct summation; leaves are always taken particle by particle
 *     (optionally, a cell that contains the particle is always opened);
 *   - optional alternative size in that test (Section V names alternative
 *     ways of computing the criterion as future work): b_max, the distance
 *     from the centre of mass to the farthest corner of the cell, which bounds
 *     the distance of every point of the cell from the centre of mass
 *     (Salmon and Warren 1994); accept iff b_max^2 < theta^2 d^2;
 *   - keys: the bounding cube is anchored at the per-axis minimum of the FP32
 *     positions with side = the largest FP32 extent (1 if that is below 1e-30);
 *     each coordinate is quantised to 21 bits as
 *       q = clamp(floor(RN32(RN32(x - lo) * RN32(2^21 / side))), 0, 2^21 - 1)
 *     using single-precision round-to-nearest operations (this is a
 *     discretisation rule, not a precision choice), and the three 21-bit
 *     integers are interleaved into a 63-bit key, x bit most significant in
 *     each triple, so the child octant at each level is 4 qx + 2 qy + qz;
 *   - tree: classic recursive insertion (Barnes & Hut 1986): particles are
 *     inserted one at a time in input order; a leaf that receives a second
 *     particle is split, the octant chosen by the key digit of the next level;
 *     at level 21 (keys identical) the leaf keeps all its particles (a
 *     bucket, members in input order);
 *   - canonical node order: depth-first pre-order, children in octant order,
 *     which is the Morton order of (level, prefix);
 *   - integrator: kick-drift-kick leapfrog, v += a dt/2; x += v dt; rebuild
 *     the tree and recompute a; v += a dt/2.
 * All floating-point sums use Neumaier's compensated summation.
 *
 * Build: gcc -O2 -std=c11 -fPIC -shared -ffp-contract=off -fopenmp
 * (-ffp-contract=off keeps every single-precision key operation a separately
 * rounded IEEE operation on every host).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_LEVELS 21
#define OR_QMAX ((1u << OR_LEVELS) - 1u)

/* ------------------------------------------------------------------ sums */

typedef struct { double s, c; } nsum;

static void nsum_add(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static double nsum_get(const nsum *a) { return a->s + a->c; }

/* Exposed so a test can check that compensation survives compilation. */
double oracle_nsum(int64_t n, const double *x)
{
    nsum a = {0.0, 0.0};
    for (int64_t i = 0; i < n; ++i) nsum_add(&a, x[i]);
    return nsum_get(&a);
}

/* ------------------------------------------------------------------ keys */

/* Bounding cube from the FP32 positions: lo = per-axis minimum, side = the
 * largest per-axis extent (each extent one FP32 subtraction). */
void oracle_cube(int64_t n, const double *pm, float lo[3], float *side)
{
    float mn[3] = {0, 0, 0}, mx[3] = {0, 0, 0};
    for (int64_t i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) {
            float x = (float)pm[4 * i + a];
            if (i == 0 || x < mn[a]) mn[a] = x;
            if (i == 0 || x > mx[a]) mx[a] = x;
        }
    }
    float s = 0.0f;
    for (int a = 0; a < 3; ++a) {
        float e = mx[a] - mn[a];
        if (e > s) s = e;
        lo[a] = mn[a];
    }
    if (!(s >= 1e-30f)) s = 1.0f;
    *side = s;
}

static uint32_t quantise(float x, float lo, float scale)
{
    float d = x - lo;       /* RN32 */
    float t = d * scale;    /* RN32 */
    float f = floorf(t);
    if (!(f > 0.0f)) return 0u;
    if (f >= (float)OR_QMAX) return OR_QMAX;
    return (uint32_t)f;
}

static uint64_t interleave3(uint32_t qx, uint32_t qy, uint32_t qz)
{
    uint64_t k = 0;
    for (int b = OR_LEVELS - 1; b >= 0; --b) {
        k = (k << 3) | ((uint64_t)((qx >> b) & 1u) << 2)
                     | ((uint64_t)((qy >> b) & 1u) << 1)
                     | (uint64_t)((qz >> b) & 1u);
    }
    return k;
}

void oracle_keys(int64_t n, const double *pm, uint64_t *keys, float lo_out[3],
                 float *side_out)
{
    float lo[3], side;
    oracle_cube(n, pm, lo, &side);
    float scale = 2097152.0f / side;  /* RN32(2^21 / side) */
    for (int64_t i = 0; i < n; ++i) {
        uint32_t q[3];
        for (int a = 0; a < 3; ++a) q[a] = quantise((float)pm[4 * i + a], lo[a], scale);
        keys[i] = interleave3(q[0], q[1], q[2]);
    }
    if (lo_out) memcpy(lo_out, lo, sizeof lo);
    if (side_out) *side_out = side;
}

static int octant_at(uint64_t key, int level)  /* level 1..21 */
{
    return (int)((key >> (3 * (OR_LEVELS - level))) & 7u);
}

/* ------------------------------------------------------------------ tree */

typedef struct {
    int level;
    uint64_t prefix;       /* key >> 3 (21 - level) */
    int32_t child[8];      /* node index or -1 */
    int is_leaf;
    int64_t np;            /* particles held by a leaf */
    int64_t cap;
    int64_t *plist;        /* leaf members (input order) */
    int64_t one;           /* inline storage when np <= 1 */
    /* filled after insertion */
    int64_t first, count;  /* range in the canonical particle order */
    double m, com[3];
    double I[6];           /* second moments about com: xx, yy, zz, xy, xz, yz */
} onode;

typedef struct otree {
    int64_t n;
    const double *pm;      /* borrowed during build; copied below */
    double *x;             /* n * 4 copy: x, y, z, m */
    uint64_t *keys;        /* by input index */
    float lo[3], side;
    onode *nodes;
    int64_t nn, ncap;
    int64_t *order;        /* canonical order -> input index */
    int64_t *dfs;          /* canonical node order -> storage index */
    int64_t ndfs;
    int have_moments;      /* onode.I filled */
} otree;

static int32_t new_node(otree *t, int level, uint64_t prefix)
{
    if (t->nn == t->ncap) {
        int64_t nc = t->ncap ? 2 * t->ncap : 1024;
        onode *p = (onode *)realloc(t->nodes, (size_t)nc * sizeof(onode));
        if (!p) return -1;
        t->nodes = p;
        t->ncap = nc;
    }
    onode *d = &t->nodes[t->nn];
    memset(d, 0, sizeof *d);
    d->level = level;
    d->prefix = prefix;
    for (int c = 0; c < 8; ++c) d->child[c] = -1;
    d->is_leaf = 1;
    d->plist = NULL;     /* used only once a leaf holds more than one */
    return (int32_t)(t->nn++);
}

static int64_t *leaf_list(onode *d) { return d->cap ? d->plist : &d->one; }

static int leaf_push(onode *d, int64_t p)
{
    if (d->np == 0 && d->cap == 0) { d->one = p; d->np = 1; return 0; }
    if (d->cap == 0) {
        int64_t *l = (int64_t *)malloc(4 * sizeof(int64_t));
        if (!l) return -1;
        l[0] = d->one;
        d->plist = l;
        d->cap = 4;
    }
    if (d->np == d->cap) {
        int64_t *l = (int64_t *)realloc(d->plist, (size_t)(2 * d->cap) * sizeof(int64_t));
        if (!l) return -1;
        d->plist = l;
        d->cap *= 2;
    }
    d->plist[d->np++] = p;
    return 0;
}

/* Insert particle p below node index ni (iterative descent). */
static int insert(otree *t, int32_t ni, int64_t p)
{
    for (;;) {
        onode *d = &t->nodes[ni];
        if (d->is_leaf) {
            if (d->np == 0 || d->level == OR_LEVELS) return leaf_push(d, p);
            /* split: move the resident particle one level down */
            int64_t q = leaf_list(d)[0];
            int lvl = d->level;
            uint64_t pre = d->prefix;
            d->is_leaf = 0;
            d->np = 0;
            int oq = octant_at(t->keys[q], lvl + 1);
            int32_t c = new_node(t, lvl + 1, (pre << 3) | (uint64_t)oq);
            if (c < 0) return -1;
            t->nodes[ni].child[oq] = c;
            if (leaf_push(&t->nodes[c], q)) return -1;
            /* fall through to descend with p from this (now internal) node */
            continue;
        }
        int o = octant_at(t->keys[p], d->level + 1);
        int32_t c = d->child[o];
        if (c < 0) {
            int lvl = d->level;
            uint64_t pre = d->prefix;
            c = new_node(t, lvl + 1, (pre << 3) | (uint64_t)o);
            if (c < 0) return -1;
            t->nodes[ni].child[o] = c;
        }
        ni = c;
    }
}

/* Depth-first pre-order, children in octant order: assigns first/count, the
 * canonical particle order and the centre of mass (FP64, Neumaier). */
static void finish(otree *t, int32_t ni, int64_t *cursor)
{
    onode *d = &t->nodes[ni];
    t->dfs[t->ndfs++] = ni;
    d->first = *cursor;
    nsum m = {0, 0}, mx[3] = {{0, 0}, {0, 0}, {0, 0}};
    if (d->is_leaf) {
        int64_t *l = leaf_list(d);
        for (int64_t k = 0; k < d->np; ++k) {
            int64_t p = l[k];
            t->order[(*cursor)++] = p;
            double pm = t->x[4 * p + 3];
            nsum_add(&m, pm);
            for (int a = 0; a < 3; ++a) nsum_add(&mx[a], pm * t->x[4 * p + a]);
        }
    } else {
        for (int o = 0; o < 8; ++o) {
            int32_t c = t->nodes[ni].child[o];
            if (c < 0) continue;
            finish(t, c, cursor);
            onode *cd = &t->nodes[c];
            nsum_add(&m, cd->m);
            for (int a = 0; a < 3; ++a) nsum_add(&mx[a], cd->m * cd->com[a]);
        }
    }
    d = &t->nodes[ni];
    d->count = *cursor - d->first;
    d->m = nsum_get(&m);
    for (int a = 0; a < 3; ++a) d->com[a] = nsum_get(&mx[a]) / d->m;
}

void oracle_tree_free(otree *t)
{
    if (!t) return;
    for (int64_t i = 0; i < t->nn; ++i)
        if (t->nodes[i].cap) free(t->nodes[i].plist);
    free(t->nodes);
    free(t->x);
    free(t->keys);
    free(t->order);
    free(t->dfs);
    free(t);
}

/* Builds the tree of n particles given as pm[4 i + {0,1,2,3}] = x, y, z, m.
 * Positions are rounded to FP32 for the key rule only.  Returns NULL when
 * n < 1, a mass is not positive, or memory runs out. */
otree *oracle_tree_build(int64_t n, const double *pm)
{
    if (n < 1) return NULL;
    for (int64_t i = 0; i < n; ++i)
        if (!(pm[4 * i + 3] > 0.0)) return NULL;
    otree *t = (otree *)calloc(1, sizeof(otree));
    if (!t) return NULL;
    t->n = n;
    t->x = (double *)malloc((size_t)n * 4 * sizeof(double));
    t->keys = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    t->order = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!t->x || !t->keys || !t->order) { oracle_tree_free(t); return NULL; }
    memcpy(t->x, pm, (size_t)n * 4 * sizeof(double));
    oracle_keys(n, pm, t->keys, t->lo, &t->side);
    int32_t root = new_node(t, 0, 0);
    if (root < 0) { oracle_tree_free(t); return NULL; }
    for (int64_t p = 0; p < n; ++p)
        if (insert(t, root, p)) { oracle_tree_free(t); return NULL; }
    t->dfs = (int64_t *)malloc((size_t)t->nn * sizeof(int64_t));
    if (!t->dfs) { oracle_tree_free(t); return NULL; }
    int64_t cursor = 0;
    finish(t, root, &cursor);
    return t;
}

int64_t oracle_tree_nnodes(const otree *t) { return t->ndfs; }

void oracle_tree_cube(const otree *t, float lo[3], float *side)
{
    memcpy(lo, t->lo, sizeof t->lo);
    *side = t->side;
}

/* Canonical node list (depth-first pre-order).  childmask bit o is set when
 * the child in octant o exists. */
void oracle_tree_export(const otree *t, int32_t *level, uint64_t *prefix,
                        int64_t *first, int64_t *count, int32_t *childmask,
                        double *mass, double *com)
{
    for (int64_t k = 0; k < t->ndfs; ++k) {
        const onode *d = &t->nodes[t->dfs[k]];
        if (level) level[k] = d->level;
        if (prefix) prefix[k] = d->prefix;
        if (first) first[k] = d->first;
        if (count) count[k] = d->count;
        if (childmask) {
            int cm = 0;
            for (int o = 0; o < 8; ++o)
                if (!d->is_leaf && d->child[o] >= 0) cm |= 1 << o;
            childmask[k] = cm;
        }
        if (mass) mass[k] = d->m;
        if (com) for (int a = 0; a < 3; ++a) com[3 * k + a] = d->com[a];
    }
}

/* order[k] = input index of the k-th particle in canonical order;
 * keys[i] = key of input particle i. */
void oracle_tree_order(const otree *t, int64_t *order, uint64_t *keys)
{
    if (order) memcpy(order, t->order, (size_t)t->n * sizeof(int64_t));
    if (keys) memcpy(keys, t->keys, (size_t)t->n * sizeof(uint64_t));
}

/* Second moments of every cell about its centre of mass, by their definition
 * I_ab = sum_j m_j (x_j - com)_a (x_j - com)_b over the member particles
 * (used by the quadrupole term of the walk). */
static void second_moments(otree *t)
{
    if (t->have_moments) return;
    for (int64_t k = 0; k < t->ndfs; ++k) {
        onode *d = &t->nodes[t->dfs[k]];
        nsum I[6];
        memset(I, 0, sizeof I);
        for (int64_t q = d->first; q < d->first + d->count; ++q) {
            int64_t p = t->order[q];
            double m = t->x[4 * p + 3];
            double r0 = t->x[4 * p] - d->com[0], r1 = t->x[4 * p + 1] - d->com[1],
                   r2 = t->x[4 * p + 2] - d->com[2];
            nsum_add(&I[0], m * r0 * r0);
            nsum_add(&I[1], m * r1 * r1);
            nsum_add(&I[2], m * r2 * r2);
            nsum_add(&I[3], m * r0 * r1);
            nsum_add(&I[4], m * r0 * r2);
            nsum_add(&I[5], m * r1 * r2);
        }
        for (int a = 0; a < 6; ++a) d->I[a] = nsum_get(&I[a]);
    }
    t->have_moments = 1;
}

/* ------------------------------------------------------------------ walk */

typedef struct {
    const otree *t;
    double G, eps2, theta2;
    int64_t self;
    int open_inside;  /* never accept a cell that contains the particle */
    int quad;         /* add each accepted cell's quadrupole term */
    int bmax;         /* the cell's size in the test is b_max, not s */
    double xi[3];
    nsum a[3], phi;
    int64_t count;
} walker;

static void term(walker *w, double m, const double *xj, int is_self)
{
    double dx = xj[0] - w->xi[0], dy = xj[1] - w->xi[1], dz = xj[2] - w->xi[2];
    double r2 = dx * dx + dy * dy + dz * dz + w->eps2;
    w->count++;
    if (r2 == 0.0) return;
    double r = sqrt(r2);
    double inv3 = 1.0 / (r2 * r);
    nsum_add(&w->a[0], m * dx * inv3);
    nsum_add(&w->a[1], m * dy * inv3);
    nsum_add(&w->a[2], m * dz * inv3);
    if (!is_self) nsum_add(&w->phi, -m / r);
}

/* The second-order term of an accepted cell: the softened kernel
 * g = 1/sqrt(|d|^2 + eps^2), d = com - x_i, expanded about the centre of mass
 * to second order in the member offsets,
 *   sum_j m_j g(d + r_j) ~ M g(d) + (1/2) I_ab d_a d_b g(d)   (sum_j m_j r_j = 0),
 * with Hessian H_ab = 3 d_a d_b / s^5 - delta_ab / s^3, s^2 = |d|^2 + eps^2.
 * Potential: -(1/2) I:H.  Acceleration: minus the gradient with respect to
 * x_i, i.e. the d-gradient of (1/2) I:H:
 *   -3 (I d) / s^5 + (15/2) (d.I.d) d / s^7 - (3/2) tr(I) d / s^5. */
static void quad_term(walker *w, const onode *d)
{
    double dx = d->com[0] - w->xi[0], dy = d->com[1] - w->xi[1], dz = d->com[2] - w->xi[2];
    double s2 = dx * dx + dy * dy + dz * dz + w->eps2;
    if (s2 == 0.0) return;
    double s = sqrt(s2);
    double s3 = s2 * s, s5 = s3 * s2, s7 = s5 * s2;
    const double *I = d->I;
    double Id0 = I[0] * dx + I[3] * dy + I[4] * dz;
    double Id1 = I[3] * dx + I[1] * dy + I[5] * dz;
    double Id2 = I[4] * dx + I[5] * dy + I[2] * dz;
    double dId = dx * Id0 + dy * Id1 + dz * Id2;
    double tr = I[0] + I[1] + I[2];
    double c = 7.5 * dId / s7 - 1.5 * tr / s5;
    nsum_add(&w->a[0], -3.0 * Id0 / s5 + c * dx);
    nsum_add(&w->a[1], -3.0 * Id1 / s5 + c * dy);
    nsum_add(&w->a[2], -3.0 * Id2 / s5 + c * dz);
    nsum_add(&w->phi, -0.5 * (3.0 * dId / s5 - tr / s3));
}

/* b_max^2 of a cell: the squared distance from its centre of mass to the
 * farthest corner of its cube.  Per axis the cube is [c, c + s] with
 * c = lo + q s, q the cell's integer position at its level (the key prefix
 * de-interleaved: bit 2 of each octal digit is x, bit 1 y, bit 0 z), and the
 * farther face is max(com - c, (c + s) - com). */
static double cell_bmax2(const otree *t, const onode *d)
{
    double s = ldexp((double)t->side, -d->level);
    uint64_t q[3] = {0, 0, 0};
    for (int b = 0; b < d->level; ++b) {
        unsigned digit = (unsigned)((d->prefix >> (3 * b)) & 7u);
        q[0] |= (uint64_t)((digit >> 2) & 1u) << b;
        q[1] |= (uint64_t)((digit >> 1) & 1u) << b;
        q[2] |= (uint64_t)(digit & 1u) << b;
    }
    double e2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double c = (double)t->lo[a] + (double)q[a] * s;
        double lo_gap = d->com[a] - c, hi_gap = (c + s) - d->com[a];
        double e = lo_gap > hi_gap ? lo_gap : hi_gap;
        e2 += e * e;
    }
    return e2;
}

static void walk(walker *w, int32_t ni)
{
    const otree *t = w->t;
    const onode *d = &t->nodes[ni];
    if (d->is_leaf) {
        const int64_t *l = d->cap ? d->plist : &d->one;
        for (int64_t k = 0; k < d->np; ++k) {
            int64_t p = l[k];
            term(w, t->x[4 * p + 3], &t->x[4 * p], p == w->self);
        }
        return;
    }
    double dx = d->com[0] - w->xi[0], dy = d->com[1] - w->xi[1], dz = d->com[2] - w->xi[2];
    double d2 = dx * dx + dy * dy + dz * dz;
    double s = ldexp((double)t->side, -d->level);
    double r2 = w->bmax ? cell_bmax2(t, d) : s * s;
    /* the cell holds the particle iff its key starts with the cell's prefix */
    int inside = (t->keys[w->self] >> (3 * (21 - d->level))) == d->prefix;
    if (r2 < w->theta2 * d2 && !(w->open_inside && inside)) {
        term(w, d->m, d->com, 0);
        if (w->quad) quad_term(w, d);
        return;
    }
    for (int o = 0; o < 8; ++o)
        if (d->child[o] >= 0) walk(w, d->child[o]);
}

/* Accelerations (and potential, interaction count) of nt target particles
 * (input indices; NULL = all n) through the tree.  acc is nt * 3.
 * options bit 0: the alternative opening rule that never accepts a cell
 * containing the particle itself (the pure test can, for theta > 1/sqrt(3):
 * the particle's own mass then enters an approximated cell); bit 1: each
 * accepted cell adds its quadrupole (second-moment) term to the monopole;
 * bit 2: the cell's size in the opening test is b_max (cell_bmax2) instead of
 * its side, i.e. accept iff b_max^2 < theta^2 d^2. */
int oracle_accel(otree *t, double G, double eps, double theta, int64_t nt,
                 const int64_t *targets, double *acc, double *pot, int64_t *count,
                 int nthreads, int options)
{
    if (options & 2) second_moments(t);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t k = 0; k < nt; ++k) {
        int64_t i = targets ? targets[k] : k;
        walker w;
        memset(&w, 0, sizeof w);
        w.t = t;
        w.G = G;
        w.eps2 = eps * eps;
        w.theta2 = theta * theta;
        w.self = i;
        w.open_inside = (options & 1) != 0;
        w.quad = (options & 2) != 0;
        w.bmax = (options & 4) != 0;
        for (int a = 0; a < 3; ++a) w.xi[a] = t->x[4 * i + a];
        walk(&w, t->dfs[0]);
        for (int a = 0; a < 3; ++a) acc[3 * k + a] = G * nsum_get(&w.a[a]);
        if (pot) pot[k] = G * nsum_get(&w.phi);
        if (count) count[k] = w.count;
    }
    return 0;
}

/* Direct O(n^2) sum for nt targets (input indices; NULL = all n). */
int oracle_direct(int64_t n, const double *pm, double G, double eps, int64_t nt,
                  const int64_t *targets, double *acc, double *pot, int nthreads)
{
    double eps2 = eps * eps;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t k = 0; k < nt; ++k) {
        int64_t i = targets ? targets[k] : k;
        nsum a[3] = {{0, 0}, {0, 0}, {0, 0}}, phi = {0, 0};
        for (int64_t j = 0; j < n; ++j) {
            double dx = pm[4 * j] - pm[4 * i];
            double dy = pm[4 * j + 1] - pm[4 * i + 1];
            double dz = pm[4 * j + 2] - pm[4 * i + 2];
            double r2 = dx * dx + dy * dy + dz * dz + eps2;
            if (r2 == 0.0) continue;
            double r = sqrt(r2);
            double inv3 = 1.0 / (r2 * r);
            double m = pm[4 * j + 3];
            nsum_add(&a[0], m * dx * inv3);
            nsum_add(&a[1], m * dy * inv3);
            nsum_add(&a[2], m * dz * inv3);
            if (j != i) nsum_add(&phi, -m / r);
        }
        for (int c = 0; c < 3; ++c) acc[3 * k + c] = G * nsum_get(&a[c]);
        if (pot) pot[k] = G * nsum_get(&phi);
    }
    return 0;
}

/* ------------------------------------------------------------ integrator */

static int accel_all(int64_t n, const double *pm, double G, double eps, double theta,
                     double *acc, double *pot, int nthreads)
{
    otree *t = oracle_tree_build(n, pm);
    if (!t) return -1;
    oracle_accel(t, G, eps, theta, n, NULL, acc, pot, NULL, nthreads, 0);  /* monopoles */
    oracle_tree_free(t);
    return 0;
}

/* Kick-drift-kick leapfrog in FP64.  pm (n*4: x,y,z,m) and vel (n*3) are
 * updated in place; acc (n*3) must hold a(x) on entry when have_acc != 0,
 * otherwise it is computed first.  The tree is rebuilt every step. */
int oracle_leapfrog(int64_t n, double *pm, double *vel, double *acc, int have_acc,
                    double G, double eps, double theta, int nsteps, double dt,
                    int nthreads)
{
    if (!have_acc && accel_all(n, pm, G, eps, theta, acc, NULL, nthreads)) return -1;
    for (int s = 0; s < nsteps; ++s) {
        for (int64_t i = 0; i < n; ++i)
            for (int a = 0; a < 3; ++a) {
                vel[3 * i + a] += 0.5 * dt * acc[3 * i + a];
                pm[4 * i + a] += dt * vel[3 * i + a];
            }
        if (accel_all(n, pm, G, eps, theta, acc, NULL, nthreads)) return -1;
        for (int64_t i = 0; i < n; ++i)
            for (int a = 0; a < 3; ++a) vel[3 * i + a] += 0.5 * dt * acc[3 * i + a];
    }
    return 0;
}

/* Conserved quantities: out = {KE, PE, Px, Py, Pz, COMx, COMy, COMz} with
 * KE = sum m v^2 / 2, PE = sum m phi / 2 (phi from the caller), P = sum m v,
 * COM = sum m x / sum m. */
void oracle_diagnostics(int64_t n, const double *pm, const double *vel,
                        const double *phi, double out[8])
{
    nsum ke = {0, 0}, pe = {0, 0}, p[3] = {{0, 0}, {0, 0}, {0, 0}},
         mx[3] = {{0, 0}, {0, 0}, {0, 0}}, mt = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
        double m = pm[4 * i + 3];
        double v2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            v2 += vel[3 * i + a] * vel[3 * i + a];
            nsum_add(&p[a], m * vel[3 * i + a]);
            nsum_add(&mx[a], m * pm[4 * i + a]);
        }
        nsum_add(&ke, 0.5 * m * v2);
        if (phi) nsum_add(&pe, 0.5 * m * phi[i]);
        nsum_add(&mt, m);
    }
    out[0] = nsum_get(&ke);
    out[1] = nsum_get(&pe);
    for (int a = 0; a < 3; ++a) {
        out[2 + a] = nsum_get(&p[a]);
        out[5 + a] = nsum_get(&mx[a]) / nsum_get(&mt);
    }
}
