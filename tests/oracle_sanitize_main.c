/*
 * Drives every entry point of the FP64 oracle once under AddressSanitizer and
 * UndefinedBehaviorSanitizer (compiled and run by test_oracle_sanitizers.py;
 * CPU only).  The oracle source is included as one translation unit, without
 * OpenMP.  Inputs cover the degenerate shapes the tree builder has to handle:
 * one and two particles, all points equal, coincident pairs (depth-cap
 * buckets), a planar and a collinear cloud, and a random cloud; every option
 * combination of the walk is run on each.  Exit status 0 means no sanitizer
 * report and every call returned success.
 */
#include "../oracle/bh_oracle.c"

#include <stdio.h>

/* splitmix64: a fixed, self-contained stream for the test's points */
static uint64_t mix_state = 0x9e3779b97f4a7c15ull;
static double uniform01(void)
{
    uint64_t z = (mix_state += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

static int exercise(const char *name, int64_t n, double *pm)
{
    float lo[3], side;
    uint64_t *keys = malloc((size_t)n * sizeof *keys);
    /* room for the two-target call below even when n = 1 */
    double *acc = malloc((size_t)(n + 2) * 3 * sizeof *acc), *pot = malloc((size_t)n * sizeof *pot);
    double *vel = calloc((size_t)n * 3, sizeof *vel);
    int64_t *cnt = malloc((size_t)n * sizeof *cnt), *order = malloc((size_t)n * sizeof *order);
    if (!keys || !acc || !pot || !vel || !cnt || !order) return 1;
    oracle_cube(n, pm, lo, &side);
    oracle_keys(n, pm, keys, lo, &side);
    otree *t = oracle_tree_build(n, pm);
    if (!t) {
        fprintf(stderr, "%s: tree build failed\n", name);
        return 1;
    }
    int64_t m = oracle_tree_nnodes(t);
    int32_t *level = malloc((size_t)m * sizeof *level), *cm = malloc((size_t)m * sizeof *cm);
    uint64_t *prefix = malloc((size_t)m * sizeof *prefix);
    int64_t *first = malloc((size_t)m * sizeof *first), *count = malloc((size_t)m * sizeof *count);
    double *mass = malloc((size_t)m * sizeof *mass), *com = malloc((size_t)m * 3 * sizeof *com);
    if (!level || !cm || !prefix || !first || !count || !mass || !com) return 1;
    oracle_tree_export(t, level, prefix, first, count, cm, mass, com);
    oracle_tree_order(t, order, keys);
    oracle_tree_cube(t, lo, &side);
    const double thetas[3] = {0.0, 0.5, 1.0};
    for (int k = 0; k < 3; ++k)
        for (int opt = 0; opt < 8; ++opt)
            if (oracle_accel(t, 1.0, 0.01, thetas[k], n, NULL, acc, pot, cnt, 1, opt)) {
                fprintf(stderr, "%s: accel failed (theta %g, options %d)\n", name, thetas[k], opt);
                return 1;
            }
    const int64_t targets[2] = {0, n - 1};
    if (oracle_accel(t, 1.0, 0.0, 0.7, 2, targets, acc, NULL, NULL, 1, 7)) return 1;
    oracle_tree_free(t);
    if (oracle_direct(n, pm, 1.0, 0.01, n, NULL, acc, pot, 1)) return 1;
    if (oracle_leapfrog(n, pm, vel, acc, 0, 1.0, 0.01, 0.5, 2, 1e-3, 1)) return 1;
    double d[8];
    oracle_diagnostics(n, pm, vel, pot, d);
    oracle_diagnostics(n, pm, vel, NULL, d);
    (void)oracle_nsum(n, pot);
    free(keys); free(acc); free(pot); free(vel); free(cnt); free(order);
    free(level); free(cm); free(prefix); free(first); free(count); free(mass); free(com);
    printf("%s: n=%lld nodes=%lld ok\n", name, (long long)n, (long long)m);
    return 0;
}

int main(void)
{
    enum { N = 300 };
    static double pm[4 * N];
    int bad = 0;
    /* one particle, two particles */
    pm[0] = 0.25; pm[1] = -0.5; pm[2] = 1.0; pm[3] = 1.0;
    bad |= exercise("one", 1, pm);
    pm[4] = -0.75; pm[5] = 0.5; pm[6] = 0.0; pm[7] = 2.0;
    bad |= exercise("two", 2, pm);
    /* all equal */
    for (int i = 0; i < 40; ++i) {
        pm[4 * i] = 0.3; pm[4 * i + 1] = 0.3; pm[4 * i + 2] = 0.3; pm[4 * i + 3] = 1.0 / 40;
    }
    bad |= exercise("all-equal", 40, pm);
    /* random cloud with coincident pairs, planar, collinear */
    for (int shape = 0; shape < 3; ++shape) {
        for (int i = 0; i < N; ++i) {
            double *p = &pm[4 * i];
            for (int a = 0; a < 3; ++a) p[a] = 2.0 * uniform01() - 1.0;
            if (shape >= 1) p[2] = 0.125;              /* planar */
            if (shape == 2) p[1] = 0.5 * p[0];         /* collinear */
            p[3] = (0.5 + uniform01()) / N;
            if (i % 7 == 3) {                          /* coincident with its predecessor */
                p[0] = p[-4]; p[1] = p[-3]; p[2] = p[-2];
            }
            /* keep the key rule's FP32 view of the inputs */
            for (int a = 0; a < 3; ++a) p[a] = (double)(float)p[a];
        }
        static const char *names[3] = {"random+pairs", "planar", "collinear"};
        bad |= exercise(names[shape], N, pm);
    }
    return bad;
}
