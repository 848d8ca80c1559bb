"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: hand-derived
values, closed forms, invariants, brute force on tiny inputs, or a textbook
special case.  Paper references: Section I (one particle per leaf, centre of
mass per cube), Section III and Fig. 1 (opening criterion), Fig. 2 (worked
example).  No GPU needed.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _pm(points, masses=None):
    p = np.asarray(points, dtype=np.float64)
    n = p.shape[0]
    pm = np.zeros((n, 4))
    pm[:, :p.shape[1]] = p
    pm[:, 3] = 1.0 / n if masses is None else masses
    return pm


# ----------------------------------------------------------------- summation

def test_neumaier_compensation_survives_compilation(oracle_lib):
    # Naive left-to-right summation returns 0 and 0 for these; the exact sums are 1 and 2.
    assert oracle.nsum([1e16, 1.0, -1e16]) == 1.0
    assert oracle.nsum([1.0, 1e100, 1.0, -1e100]) == 2.0


# ---------------------------------------------------------------------- keys

def test_keys_hand_derived(oracle_lib):
    with open(os.path.join(GOLDEN, "keys_hand.json")) as f:
        cases = json.load(f)["cases"]
    for case in cases:
        k = oracle.keys(_pm(case["points"]))
        assert [int(x) for x in k] == [int(x) for x in case["keys"]], case["name"]


def test_key_octant_matches_geometry(oracle_lib):
    # Level-1 octant = 4*[x in upper half] + 2*[y upper] + [z upper] (x most significant).
    rng = np.random.default_rng(7)
    p = rng.uniform(-3, 5, (500, 3))
    pm = _pm(np.vstack([p, [[-3, -3, -3], [5, 5, 5]]]))  # pin the cube to [-3, 5]^3
    k = oracle.keys(pm)
    oct1 = (k >> np.uint64(60)).astype(int)
    mid = 1.0
    want = 4 * (pm[:, 0] >= mid) + 2 * (pm[:, 1] >= mid) + (pm[:, 2] >= mid)
    far = np.all(np.abs(pm[:, :3] - mid) > 1e-5, axis=1)
    assert np.array_equal(oct1[far], want[far])


def test_key_rule_rounds_in_single_precision(oracle_lib):
    # The rule quantises with FP32 round-to-nearest operations.  numpy float32
    # arithmetic is an independent IEEE implementation of the same operations;
    # we look for points where exact (FP64) arithmetic would give another
    # integer and check the oracle follows the FP32 rule there.
    rng = np.random.default_rng(11)
    x = rng.uniform(-1, 1, 200000).astype(np.float32)
    lo = np.float32(-1.0)
    side = np.float32(2.0)
    scale = np.float32(2097152.0) / side
    q32 = np.floor((x - lo) * scale).astype(np.int64)
    q64 = np.floor((x.astype(np.float64) + 1.0) * 2097152.0 / 2.0).astype(np.int64)
    differ = np.nonzero(q32 != q64)[0]
    assert differ.size > 0
    pts = np.zeros((differ.size + 2, 3))
    pts[:-2, 0] = x[differ]
    pts[-2] = [-1, -1, -1]
    pts[-1] = [1, 1, 1]
    k = oracle.keys(_pm(pts))[:-2]
    # de-interleave qx from the key
    qx = np.zeros(k.size, np.int64)
    for b in range(21):
        qx |= ((k >> np.uint64(3 * b + 2)) & np.uint64(1)).astype(np.int64) << b
    assert np.array_equal(qx, np.clip(q32[differ], 0, 2 ** 21 - 1))


# ------------------------------------------------------------------ topology

def _brute_force_nodes(pm):
    """Every (level, prefix) cell by enumeration: a cell is a node iff it is the
    root or its parent cell holds >= 2 particles (and the parent is above the
    depth cap); sorted into depth-first Morton order."""
    k = oracle.keys(pm)
    n = len(k)
    order = np.lexsort((np.arange(n), k))  # key, then input index
    ks = k[order]
    nodes = []
    for lvl in range(22):
        pref = ks >> np.uint64(3 * (21 - lvl))
        parent = ks >> np.uint64(3 * (21 - lvl + 1)) if lvl > 0 else None
        starts = [0] + [i for i in range(1, n) if pref[i] != pref[i - 1]]
        for a, s in enumerate(starts):
            e = starts[a + 1] if a + 1 < len(starts) else n
            if lvl > 0:
                pc = np.count_nonzero(parent == parent[s])
                if pc < 2:
                    continue
            nodes.append((int(pref[s]) << (3 * (21 - lvl)), lvl, int(pref[s]), s, e - s))
    nodes.sort()
    out = []
    for i, (_, lvl, pre, first, cnt) in enumerate(nodes):
        cm = 0
        if cnt > 1 and lvl < 21:
            for (_, l2, p2, f2, c2) in nodes:
                if l2 == lvl + 1 and (p2 >> 3) == pre:
                    cm |= 1 << (p2 & 7)
        out.append((lvl, pre, first, cnt, cm))
    return out, order


@pytest.mark.parametrize("kind,n,seed", [
    ("gauss", 1, 1), ("gauss", 2, 2), ("gauss", 17, 3), ("planar", 33, 4),
    ("clustered", 48, 5), ("line", 40, 6), ("gauss", 64, 7), ("dups", 30, 8),
])
def test_topology_recursive_insertion_equals_enumeration(oracle_lib, kind, n, seed):
    if kind == "dups":
        pm, _ = synth.random_cloud(n, seed, "gauss")
        pm = pm.astype(np.float64)
        pm[5:12, :3] = pm[3, :3]      # a bucket of 8 coincident points
        pm[20:23, :3] = pm[19, :3]
    else:
        pm, _ = synth.random_cloud(n, seed, kind)
    T = oracle.Tree(pm)
    nd = T.nodes()
    got = list(zip(nd["level"].tolist(), nd["prefix"].tolist(), nd["first"].tolist(),
                   nd["count"].tolist(), nd["childmask"].tolist()))
    want, order = _brute_force_nodes(pm.astype(np.float64))
    assert got == want
    o, _ = T.order()
    assert np.array_equal(o, order)


def test_topology_hand_cases(oracle_lib):
    with open(os.path.join(GOLDEN, "topology_hand.json")) as f:
        cases = json.load(f)["cases"]
    for case in cases:
        T = oracle.Tree(_pm(case["points"]))
        nd = T.nodes()
        got = [[int(nd["level"][i]), int(nd["prefix"][i]), int(nd["first"][i]),
                int(nd["count"][i]), int(nd["childmask"][i])] for i in range(T.m)]
        assert got == case["nodes"], case["name"]
        o, _ = T.order()
        assert o.tolist() == case["order"], case["name"]


# ----------------------------------------------------------- centre of mass

def test_com_invariants(oracle_lib):
    pm, _ = synth.random_cloud(3000, 21, "clustered")
    pm = pm.astype(np.float64)
    T = oracle.Tree(pm)
    nd = T.nodes()
    o, _ = T.order()
    m = pm[o, 3]
    x = pm[o, :3]
    # root: total mass and mass-weighted mean
    assert nd["level"][0] == 0
    assert abs(nd["mass"][0] - m.sum()) <= 1e-14 * m.sum()
    np.testing.assert_allclose(nd["com"][0], (m[:, None] * x).sum(0) / m.sum(), rtol=0,
                               atol=1e-14 * np.abs(x).max())
    # every node: mass and centre of its member particles
    cs = np.concatenate([[0.0], np.cumsum(m)])
    for i in range(T.m):
        f, c = nd["first"][i], nd["count"][i]
        mm = m[f:f + c].sum()
        assert abs(nd["mass"][i] - mm) <= 1e-13 * mm
        com = (m[f:f + c, None] * x[f:f + c]).sum(0) / mm
        np.testing.assert_allclose(nd["com"][i], com, rtol=0, atol=1e-12 * (1 + np.abs(com).max()))


# ---------------------------------------------------------------------- force

def test_direct_sum_two_body_closed_form(oracle_lib):
    # |a_1| = G m_2 / r^2 exactly, pointing at body 2 (eps = 0).
    pm = _pm([[0.3, -0.2, 0.1], [1.3, 0.8, -0.4]], [2.0, 0.5])
    acc, pot = oracle.direct(pm, eps=0.0, G=1.7)
    r = np.array([1.0, 1.0, -0.5])
    rr = np.linalg.norm(r)
    np.testing.assert_allclose(acc[0], 1.7 * 0.5 * r / rr ** 3, rtol=1e-15)
    np.testing.assert_allclose(acc[1], -1.7 * 2.0 * r / rr ** 3, rtol=1e-15)
    np.testing.assert_allclose(pot, [-1.7 * 0.5 / rr, -1.7 * 2.0 / rr], rtol=1e-15)


def test_direct_sum_cube_vertices_closed_form(oracle_lib):
    # 8 unit masses on the vertices of [-1,1]^3.  The pull on (1,1,1) points
    # along -(1,1,1)/sqrt3 with magnitude 3/(4 sqrt3) + (3/8) sqrt(2/3) + 1/12
    # (three edge neighbours at 2, three face diagonals at 2 sqrt2, one body
    # diagonal at 2 sqrt3), derived by hand.
    v = np.array([[x, y, z] for x in (-1, 1) for y in (-1, 1) for z in (-1, 1)], float)
    acc, pot = oracle.direct(_pm(v, np.ones(8)), eps=0.0)
    mag = 3 / (4 * math.sqrt(3)) + (3 / 8) * math.sqrt(2 / 3) + 1 / 12
    i = 7  # (1,1,1)
    np.testing.assert_allclose(acc[i], -mag / math.sqrt(3) * np.ones(3), rtol=1e-14)
    np.testing.assert_allclose(pot[i], -(3 / 2 + 3 / (2 * math.sqrt(2)) + 1 / (2 * math.sqrt(3))),
                               rtol=1e-14)


def test_theta_zero_is_direct_summation(oracle_lib):
    # theta = 0 never accepts a cell, so the walk is the direct sum; the gate is
    # max_i |a_tree - a_direct| / sum_j |G m_j r_ij|/(r^2+eps^2)^(3/2) <= 1e-12.
    pm, _ = synth.plummer(1500, 1)
    pm = pm.astype(np.float64)
    eps = 0.01
    at, pt, cnt = oracle.Tree(pm).accel(0.0, eps)
    ad, pd = oracle.direct(pm, eps)
    x, m = pm[:, :3], pm[:, 3]
    r = x[None, :, :] - x[:, None, :]
    r2 = (r ** 2).sum(-1) + eps ** 2
    scale = (m[None, :] * np.sqrt((r ** 2).sum(-1)) / r2 ** 1.5).sum(1)
    assert (np.abs(at - ad).max(1) / scale).max() <= 1e-12
    assert np.all(cnt == len(pm))  # every particle individually


def test_momentum_conserved_by_pairwise_sums(oracle_lib):
    pm, _ = synth.random_cloud(700, 3, "gauss")
    pm = pm.astype(np.float64)
    m = pm[:, 3]
    for acc in (oracle.direct(pm, 0.05)[0], oracle.Tree(pm).accel(0.0, 0.05)[0]):
        tot = (m[:, None] * acc).sum(0)
        assert np.abs(tot).max() <= 1e-13 * (m[:, None] * np.abs(acc)).sum()


def test_error_decreases_as_theta_decreases(oracle_lib):
    pm, _ = synth.plummer(3000, 2)
    pm = pm.astype(np.float64)
    ad, _ = oracle.direct(pm, 0.01)
    T = oracle.Tree(pm)
    errs = []
    for th in (1.0, 0.7, 0.5, 0.3, 0.15):
        a, _, _ = T.accel(th, 0.01)
        errs.append(np.median(np.linalg.norm(a - ad, axis=1) / np.linalg.norm(ad, axis=1)))
    assert all(e1 > e2 for e1, e2 in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-4


def _quantised(x, lo, side):
    """Level-21 integer position of each point by the key rule, in numpy FP32
    arithmetic (independent of the oracle's key code)."""
    scale = np.float32(2097152.0) / np.float32(side)
    q = np.floor((x.astype(np.float32) - np.asarray(lo, np.float32)) * scale).astype(np.int64)
    return np.clip(q, 0, 2 ** 21 - 1)


def _frontier_accel(pm, theta, eps, lo_side, open_inside=False, bmax=False):
    """The Barnes-Hut sum from its set definition, without recursion: particle
    i uses every node whose proper ancestors all fail the opening test s^2 <
    theta^2 d^2 for i while the node itself passes it, is a one-particle leaf,
    or is a depth-cap bucket (then each member particle).  Nodes by brute-force
    enumeration; centres of mass as direct sums over member particles.
    bmax: the test's s is the largest distance from the centre of mass to one
    of the cell's 8 corners (all enumerated), the cell placed by the integer
    position of its first member at the cell's level."""
    nodes, order = _brute_force_nodes(pm)
    keys_sorted = oracle.keys(pm)[order]
    x = pm[order, :3]
    m = pm[order, 3]
    side = float(lo_side[1])
    lo = np.asarray(lo_side[0], np.float32).astype(np.float64)
    q21 = _quantised(x, lo_side[0], lo_side[1])
    com = {}
    for (lvl, pre, first, cnt, _) in nodes:
        mm = m[first:first + cnt]
        com[(lvl, pre)] = (mm.sum(), (mm[:, None] * x[first:first + cnt]).sum(0) / mm.sum())
    n = len(pm)
    acc = np.zeros((n, 3)); pot = np.zeros(n); count = np.zeros(n, np.int64)
    for i in range(n):
        xi = x[i]

        key_i = int(keys_sorted[i])
        firsts = {(lvl, pre): first for (lvl, pre, first, cnt, _) in nodes}

        def opens(lvl, pre, cnt):
            if cnt == 1 or lvl == 21:
                return False
            if open_inside and (key_i >> (3 * (21 - lvl))) == pre:
                return True
            M, c = com[(lvl, pre)]
            s = side * 2.0 ** -lvl
            if bmax:
                c0 = lo + (q21[firsts[(lvl, pre)]] >> (21 - lvl)) * s
                r2 = max(float(((c0 + np.array(b) * s - c) ** 2).sum())
                         for b in itertools.product((0.0, 1.0), repeat=3))
            else:
                r2 = s * s
            return not (r2 < theta * theta * float(((c - xi) ** 2).sum()))

        info = {(lvl, pre): cnt for (lvl, pre, first, cnt, _) in nodes}
        for (lvl, pre, first, cnt, _) in nodes:
            if opens(lvl, pre, cnt):
                continue
            if not all(opens(l2, pre >> (3 * (lvl - l2)), info[(l2, pre >> (3 * (lvl - l2)))])
                       for l2 in range(lvl)):
                continue
            members = range(first, first + cnt) if (cnt == 1 or lvl == 21) else None
            terms = [(m[j], x[j], j == i) for j in members] if members is not None else \
                [(com[(lvl, pre)][0], com[(lvl, pre)][1], False)]
            for (mj, xj, self_term) in terms:
                d = xj - xi
                r2 = float((d ** 2).sum()) + eps * eps
                count[i] += 1
                if r2 > 0.0:
                    acc[i] += mj * d / r2 ** 1.5
                    if not self_term:
                        pot[i] -= mj / np.sqrt(r2)
    out_a = np.zeros_like(acc); out_p = np.zeros_like(pot); out_c = np.zeros_like(count)
    out_a[order] = acc; out_p[order] = pot; out_c[order] = count
    return out_a, out_p, out_c


@pytest.mark.parametrize("rule", ["pure", "open_inside", "bmax", "bmax+open_inside"])
@pytest.mark.parametrize("kind,n,seed", [("gauss", 40, 11), ("clustered", 60, 12),
                                         ("planar", 50, 13), ("dups", 30, 14)])
@pytest.mark.parametrize("theta", [0.3, 0.5, 0.7, 1.0])
def test_walk_equals_set_definition(oracle_lib, kind, n, seed, theta, rule):
    # theta > 0: the recursive walk against the set definition of the sum it
    # computes, on inputs small enough to enumerate every node and ancestor
    if kind == "dups":
        pm, _ = synth.random_cloud(n, seed, "gauss")
        pm = pm.astype(np.float64)
        pm[4:10, :3] = pm[2, :3]      # a bucket of 7 coincident points
    else:
        pm, _ = synth.random_cloud(n, seed, kind)
        pm = pm.astype(np.float64)
    pm[:, 3] *= np.linspace(0.5, 1.5, n)  # unequal masses: a centroid is not the COM
    eps = 0.01
    open_inside, bmax = "open_inside" in rule, "bmax" in rule
    T = oracle.Tree(pm)
    a, p, c = T.accel(theta, eps, open_inside=open_inside, bmax=bmax)
    lo, side = T.cube()
    wa, wp, wc = _frontier_accel(pm, theta, eps, (lo, side), open_inside, bmax)
    assert np.array_equal(c, wc)
    scale = np.abs(wa).max()
    assert np.abs(a - wa).max() <= 1e-12 * scale
    assert np.abs(p - wp).max() <= 1e-12 * np.abs(wp).max()


def test_fig2_two_inputs_for_remote_particles(oracle_lib):
    # Fig. 2 (Section III): four particles in a 2-D domain; P3 and P4 cluster in
    # node N2, so P1 and P2 each need only two inputs (the other remote
    # particle and N2's centroid).  Counts below exclude the self term.
    with open(os.path.join(GOLDEN, "fig2_shape.json")) as f:
        g = json.load(f)
    pm = _pm(g["points"])
    _, _, cnt = oracle.Tree(pm).accel(g["theta"], g["eps"])
    assert (cnt - 1).tolist() == g["inputs_excluding_self"]


# --------------------------------------------------------------- integrator

def test_leapfrog_kepler_orbit_second_order(oracle_lib):
    pm, vel, k = synth.kepler_pair(0.6, 0.4, 1.0, 0.5)
    x0 = pm.astype(np.float64)
    T = k["period"]
    errs = []
    for nsteps in (500, 1000, 2000):
        p, v, _ = oracle.leapfrog(x0, vel, nsteps, T / nsteps, theta=0.5, eps=0.0)
        errs.append(np.abs(p[:, :3] - x0[:, :3]).max())
    # KDK is second order: halving dt divides the one-orbit error by ~4.
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0, errs
    assert errs[-1] < 1e-3


def test_leapfrog_kepler_energy_and_reversibility(oracle_lib):
    pm, vel, k = synth.kepler_pair(0.6, 0.4, 1.0, 0.5)
    x0 = pm.astype(np.float64)
    dt = k["period"] / 1000
    p, v, a = oracle.leapfrog(x0, vel, 1000, dt, theta=0.5, eps=0.0)
    e0 = 0.5 * 0.6 * (vel[0, :3].astype(float) ** 2).sum() + 0.5 * 0.4 * (vel[1, :3].astype(float) ** 2).sum() \
        - 0.6 * 0.4 / k["rp"]
    e1 = 0.5 * 0.6 * (v[0] ** 2).sum() + 0.5 * 0.4 * (v[1] ** 2).sum() \
        - 0.6 * 0.4 / np.linalg.norm(p[0, :3] - p[1, :3])
    assert abs(e1 - e0) < 1e-4 * abs(e0)
    # run backwards: the scheme is time-reversible
    pb, vb, _ = oracle.leapfrog(p, -v, 1000, dt, theta=0.5, eps=0.0, acc=a)
    np.testing.assert_allclose(pb[:, :3], x0[:, :3], atol=1e-10)


def test_diagnostics_hand_values(oracle_lib):
    pm = _pm([[1.0, 0, 0], [-1.0, 0, 0], [0, 2.0, 0]], [1.0, 2.0, 3.0])
    vel = np.array([[0, 1.0, 0], [0, 0, 2.0], [3.0, 0, 0]])
    phi = np.array([-1.0, -2.0, -3.0])
    d = oracle.diagnostics(pm, vel, phi)
    # KE = 0.5(1*1 + 2*4 + 3*9) = 18; PE = 0.5(-1 - 4 - 9) = -7
    # P = (9, 1, 4); COM = (1 - 2 + 0, 6, 0)/6
    np.testing.assert_allclose(d, [18.0, -7.0, 9.0, 1.0, 4.0, -1 / 6, 1.0, 0.0], rtol=1e-15)


# ----------------------------------------------------------- input recipe

def test_plummer_generator_matches_model(oracle_lib):
    # Half-mass radius of the a=1 Plummer sphere is (2^(2/3) - 1)^(-1/2) = 1.3048;
    # virial equilibrium: 2 KE + PE = 0 with KE = 3 pi/64, PE = -3 pi/32 (G=M=a=1).
    pm, vel = synth.plummer(100000, 9)
    r = np.sort(np.linalg.norm(pm[:, :3].astype(np.float64), axis=1))
    assert abs(r[len(r) // 2] - 1.3048) < 0.03
    assert abs(pm[:, 3].astype(np.float64).sum() - 1.0) < 1e-5
    pm2, vel2 = synth.plummer(4096, 10)
    _, pot = oracle.direct(pm2, 1e-4)
    d = oracle.diagnostics(pm2, vel2, pot)
    assert abs(d[0] - 3 * math.pi / 64) < 0.1 * 3 * math.pi / 64
    assert abs(2 * d[0] + d[1]) < 0.1 * abs(d[1])


def test_open_inside_changes_only_cells_holding_the_particle(oracle_lib):
    # below theta = 1/sqrt(3) a cell holding the particle always fails the
    # test (d <= sqrt(3) s), so the rule changes nothing; above it, it opens
    # such cells and so adds interactions
    pm, _ = synth.plummer(2000, 9)
    T = oracle.Tree(pm)
    for theta in (0.3, 0.5, 0.57):
        a0, p0, c0 = T.accel(theta, 0.01)
        a1, p1, c1 = T.accel(theta, 0.01, open_inside=True)
        assert np.array_equal(c0, c1) and np.array_equal(a0, a1)
    a0, _, c0 = T.accel(0.9, 0.01)
    a1, _, c1 = T.accel(0.9, 0.01, open_inside=True)
    assert np.all(c1 >= c0) and np.count_nonzero(c1 > c0) > 0


def _cluster_and_probe(D, seed=3):
    """A compact cluster of 12 unequal masses (radius ~0.05) at the origin and a
    light probe particle at distance D along a fixed direction; with theta =
    0.9 the probe accepts the cluster's cell as one body."""
    rng = np.random.default_rng(seed)
    pts = rng.normal(0.0, 0.02, size=(12, 3))
    m = rng.uniform(0.5, 1.5, 12)
    pm = np.zeros((13, 4))
    pm[:12, :3] = pts
    pm[:12, 3] = m
    u = np.array([0.48, 0.6, 0.64])
    pm[12, :3] = D * u / np.linalg.norm(u)
    pm[12, 3] = 1e-9
    return pm


def test_quadrupole_force_is_minus_gradient_of_its_potential(oracle_lib):
    # the acceleration and potential formulas of the quadrupole term are
    # written separately; a central difference of the potential at the probe
    # must reproduce the acceleration there (monopole and quadrupole together)
    pm = _cluster_and_probe(2.0)
    T = oracle.Tree(pm)
    a, _, c = T.accel(0.9, 0.01, targets=[12], quadrupole=True)
    a_mono, _, c_mono = T.accel(0.9, 0.01, targets=[12])
    assert c[0] == c_mono[0] == 1  # the whole cluster is one accepted cell
    assert np.linalg.norm(a - a_mono) > 1e-6 * np.linalg.norm(a)  # the term matters here
    h = 1e-5
    grad = np.zeros(3)
    for k in range(3):
        phis = []
        for sgn in (1.0, -1.0):
            q = pm.copy()
            q[12, k] += sgn * h
            _, phi, cc = oracle.Tree(q).accel(0.9, 0.01, targets=[12], quadrupole=True)
            assert cc[0] == 1
            phis.append(phi[0])
        grad[k] = (phis[0] - phis[1]) / (2 * h)
    np.testing.assert_allclose(a[0], -grad, rtol=1e-6)


def test_quadrupole_error_falls_one_order_faster(oracle_lib):
    # relative to the exact pull of the cluster, the monopole error falls as
    # D^-2 and the error with the quadrupole term as D^-3 (the next term of the
    # expansion); checked by log-log slopes over D = 2 .. 16
    Ds = np.array([2.0, 4.0, 8.0, 16.0])
    em, eq = [], []
    for D in Ds:
        pm = _cluster_and_probe(D)
        ad, _ = oracle.direct(pm, 0.01, targets=[12])
        T = oracle.Tree(pm)
        a0, _, _ = T.accel(0.9, 0.01, targets=[12])
        a1, _, _ = T.accel(0.9, 0.01, targets=[12], quadrupole=True)
        n = np.linalg.norm(ad[0])
        em.append(np.linalg.norm(a0[0] - ad[0]) / n)
        eq.append(np.linalg.norm(a1[0] - ad[0]) / n)
    sm = np.polyfit(np.log(Ds), np.log(em), 1)[0]
    sq = np.polyfit(np.log(Ds), np.log(eq), 1)[0]
    assert -2.3 < sm < -1.7, sm
    assert sq < -2.7, sq
    assert all(q < m for q, m in zip(eq, em))


def test_quadrupole_keeps_the_accepted_set(oracle_lib):
    pm, _ = synth.plummer(1500, 21)
    T = oracle.Tree(pm)
    for theta in (0.5, 0.8):
        _, _, c0 = T.accel(theta, 0.01)
        _, _, c1 = T.accel(theta, 0.01, quadrupole=True)
        assert np.array_equal(c0, c1)


# ------------------------------------------------------ b_max opening rule

def test_bmax_rule_between_two_pure_tests(oracle_lib):
    # every point of a cell lies within b_max of its centre of mass, and the
    # centre lies inside the cell, so sqrt(3)/2 s <= b_max <= sqrt(3) s: the
    # rule at theta accepts whatever the pure test accepts at theta/sqrt(3) and
    # nothing that it rejects at 2 theta/sqrt(3).  A rule that accepts more
    # reaches fewer, coarser nodes, so per particle
    #   count_pure(2 theta/sqrt(3)) <= count_bmax(theta) <= count_pure(theta/sqrt(3)),
    # both strict for some particles (b_max is neither bound)
    pm, _ = synth.plummer(2000, 23)
    T = oracle.Tree(pm)
    r3 = math.sqrt(3.0)
    for theta in (0.5, 0.8):
        _, _, c = T.accel(theta, 0.01, bmax=True)
        _, _, c_hi = T.accel(2 * theta / r3, 0.01)
        _, _, c_lo = T.accel(theta / r3, 0.01)
        assert np.all(c_hi <= c) and np.all(c <= c_lo)
        assert np.count_nonzero(c_hi < c) > 0 and np.count_nonzero(c < c_lo) > 0


def test_bmax_rule_never_accepts_the_particles_own_cell(oracle_lib):
    # d <= b_max for a particle inside the cell, so for theta <= 1 the rule
    # never accepts a cell that holds the particle: the open-inside rule then
    # changes nothing, while under the pure test it does at theta = 0.9, 1.0
    pm, _ = synth.plummer(2000, 24)
    T = oracle.Tree(pm)
    for theta in (0.9, 1.0):
        a0, p0, c0 = T.accel(theta, 0.01, bmax=True)
        a1, p1, c1 = T.accel(theta, 0.01, bmax=True, open_inside=True)
        assert np.array_equal(c0, c1) and np.array_equal(a0, a1) and np.array_equal(p0, p1)
        _, _, d0 = T.accel(theta, 0.01)
        _, _, d1 = T.accel(theta, 0.01, open_inside=True)
        assert np.any(d0 != d1)



# ---------------------------------------------------- many-body invariants

def _energy(pm, v, eps):
    _, phi = oracle.direct(pm, eps)
    m = pm[:, 3]
    return 0.5 * (m * (v ** 2).sum(1)).sum() + 0.5 * (m * phi).sum()


def test_leapfrog_many_body_conservation_laws(oracle_lib):
    # theta = 0 (every pair summed directly, softened central forces): total
    # momentum and angular momentum are conserved to rounding by every KDK
    # step, and the energy error of the symplectic scheme is second order in
    # dt -- halving dt quarters it -- for a Plummer sphere of 256 bodies
    pm, vel = synth.plummer(256, 31)
    pm = pm.astype(np.float64); v0 = vel[:, :3].astype(np.float64)
    eps = 0.05
    e0 = _energy(pm, v0, eps)
    m = pm[:, 3]
    p0 = (m[:, None] * v0).sum(0)
    l0 = (m[:, None] * np.cross(pm[:, :3], v0)).sum(0)
    errs = []
    for nsteps, dt in ((20, 2e-2), (40, 1e-2), (80, 5e-3)):
        p, v, _ = oracle.leapfrog(pm, vel, nsteps, dt, theta=0.0, eps=eps)
        mv = m[:, None] * v
        assert np.abs(mv.sum(0) - p0).max() < 1e-14
        assert np.abs((m[:, None] * np.cross(p[:, :3], v)).sum(0) - l0).max() < 1e-13
        errs.append(abs(_energy(p, v, eps) - e0) / abs(e0))
    assert errs[0] < 1e-3
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0, errs


def test_walk_linear_in_masses_and_G_and_independent_of_input_order(oracle_lib):
    # the tree depends on positions only, so scaling every mass by 2 and G by
    # 4 scales every acceleration and potential by exactly 8 (powers of two);
    # and the canonical tree and depth-first sum order make every particle's
    # result independent of the order the particles are given in
    pm, _ = synth.plummer(1500, 33)
    pm = pm.astype(np.float64)
    pm[:, 3] *= np.linspace(0.5, 1.5, len(pm))
    for theta in (0.0, 0.6, 1.0):
        a, p, c = oracle.Tree(pm).accel(theta, 0.01)
        q = pm.copy(); q[:, 3] *= 2.0
        a2, p2, c2 = oracle.Tree(q).accel(theta, 0.01, G=4.0)
        assert np.array_equal(c2, c) and np.array_equal(a2, 8.0 * a) and np.array_equal(p2, 8.0 * p)
        perm = np.random.default_rng(34).permutation(len(pm))
        a3, p3, c3 = oracle.Tree(pm[perm]).accel(theta, 0.01)
        assert np.array_equal(c3, c[perm]) and np.array_equal(a3, a[perm])
        assert np.array_equal(p3, p[perm])


# ---------------------------------------------------------- input recipes

def test_input_recipes_match_their_statements():
    # the seeded generators hold no method arithmetic; these check the input
    # recipes as stated: determinism per seed, the uniform cube's range and
    # masses, the forest's size law and kinds, and the request stream's rate
    # and ranges
    a1, v1 = synth.uniform_cube(4096, 3)
    a2, v2 = synth.uniform_cube(4096, 3)
    b1, _ = synth.uniform_cube(4096, 4)
    assert np.array_equal(a1, a2) and np.array_equal(v1, v2) and not np.array_equal(a1, b1)
    assert a1.dtype == np.float32 and np.abs(a1[:, :3]).max() <= 1.0
    assert np.all(a1[:, 3] == np.float32(1.0 / 4096)) and not np.any(v1[:, :3])
    p1, _ = synth.plummer(2048, 5)
    p2, _ = synth.plummer(2048, 5)
    assert np.array_equal(p1, p2)
    # forest: N log-uniform in [256, 65536]; even index Plummer, odd uniform
    fs = synth.forest_systems(512, 256, 65536, seed=4, materialise=False)
    ns = np.array([s.n for s in fs])
    assert ns.min() >= 256 and ns.max() <= 65536
    logs = np.log(ns)
    # a log-uniform law has its median at the geometric mean and the
    # variance of U(log 256, log 65536)
    assert abs(np.median(logs) - 0.5 * (np.log(256) + np.log(65536))) < 0.35
    assert abs(logs.var() - (np.log(65536 / 256)) ** 2 / 12) < 0.5
    assert all(s.kind == ("plummer" if k % 2 == 0 else "uniform") for k, s in enumerate(fs))
    # request stream: Poisson arrivals at 200/s for 60 s, N log-uniform in
    # [1024, 2097152], theta in [0.5, 0.8], 10..200 steps
    rs = synth.request_stream(200.0, 60.0, seed=5)
    t = np.array([r.arrival_s for r in rs])
    assert abs(len(rs) - 12000) < 4 * np.sqrt(12000)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 200) < 0.05 / 200 and abs(gaps.std() / gaps.mean() - 1) < 0.05
    n = np.array([r.n for r in rs])
    th = np.array([r.theta for r in rs])
    st = np.array([r.steps for r in rs])
    assert n.min() >= 1024 and n.max() <= 2097152
    assert th.min() >= 0.5 and th.max() <= 0.8 and st.min() >= 10 and st.max() <= 200
    assert abs(np.mean([r.kind == "plummer" for r in rs]) - 0.5) < 0.02
