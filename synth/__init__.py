"""Seeded synthetic inputs for the Barnes-Hut hot path.

This module is shared by the FP64 oracle's tests, the GPU parity tests and the
benchmark.  It draws particles and request schedules only: it holds none of the
method's arithmetic (no keys, no tree, no forces, no integrator).

Workloads (all seeded, numpy PCG64 generator):

* Plummer sphere -- the paper's inputs are Plummer-model globular clusters
  generated with Piet Hut's program (Section IV).  That program is not
  available, so the model is sampled here from its published distribution
  functions (Aarseth, Henon & Wielen 1974): scale radius a = 1, total mass
  M = 1, G = 1, no N-body-unit rescaling.  Radius r = (X^(-2/3) - 1)^(-1/2)
  with X ~ U(0,1) redrawn when X > 0.999 (caps r near 38.7); speed
  v = q * sqrt(2) * (1 + r^2)^(-1/4) with q drawn by von Neumann rejection
  on g(q) = q^2 (1 - q^2)^(7/2) (g <= 0.1); isotropic directions for both.
  The centre of mass and mean velocity are removed in FP64 and the result is
  rounded to FP32.
* Uniform cube -- positions U[-1, 1]^3, zero velocities ("cold collapse").
* Kepler two-body -- two point masses on a bound orbit, for closed-form tests.
* Forest -- many independent systems of log-uniform size, half Plummer and
  half uniform cube.
* Request stream -- Poisson arrivals of solves of log-uniform size.

Arrays use the library's layout: ``pos_mass`` is float32 (N, 4) = (x, y, z, m)
and ``vel`` is float32 (N, 4) = (vx, vy, vz, 0).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "plummer", "uniform_cube", "kepler_pair", "forest_systems",
    "request_stream", "random_cloud", "System", "Request",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    """Unit vectors uniform on the sphere: z ~ U(-1,1), phi ~ U(0, 2 pi)."""
    z = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)


def _pack(pos: np.ndarray, vel: np.ndarray, mass: np.ndarray):
    n = pos.shape[0]
    pm = np.zeros((n, 4), dtype=np.float32)
    pm[:, :3] = pos.astype(np.float32)
    pm[:, 3] = mass.astype(np.float32)
    v4 = np.zeros((n, 4), dtype=np.float32)
    v4[:, :3] = vel.astype(np.float32)
    return pm, v4


def plummer(n: int, seed: int, remove_com: bool = True):
    """Plummer sphere of ``n`` equal-mass (1/n) particles; see module doc."""
    n = int(n)
    if n <= 0:
        return np.zeros((0, 4), np.float32), np.zeros((0, 4), np.float32)
    rng = _rng(seed)
    # radii by inverse transform of the cumulative mass M(r) = r^3/(1+r^2)^(3/2)
    x = np.empty(0)
    while x.size < n:
        cand = rng.uniform(0.0, 1.0, 2 * (n - x.size) + 16)
        cand = cand[(cand > 0.0) & (cand <= 0.999)]
        x = np.concatenate([x, cand])
    x = x[:n]
    r = 1.0 / np.sqrt(np.power(x, -2.0 / 3.0) - 1.0)
    pos = r[:, None] * _isotropic(rng, n)
    # speeds by rejection on g(q) = q^2 (1-q^2)^3.5, bounded by 0.1
    q = np.empty(0)
    while q.size < n:
        m = 2 * (n - q.size) + 16
        qq = rng.uniform(0.0, 1.0, m)
        yy = rng.uniform(0.0, 0.1, m)
        q = np.concatenate([q, qq[yy < qq * qq * np.power(1.0 - qq * qq, 3.5)]])
    q = q[:n]
    speed = q * math.sqrt(2.0) * np.power(1.0 + r * r, -0.25)
    vel = speed[:, None] * _isotropic(rng, n)
    if remove_com:
        pos = pos - pos.mean(axis=0)
        vel = vel - vel.mean(axis=0)
    mass = np.full(n, 1.0 / n)
    return _pack(pos, vel, mass)


def uniform_cube(n: int, seed: int, half: float = 1.0):
    """``n`` particles U[-half, half]^3, zero velocity, masses 1/n."""
    n = int(n)
    rng = _rng(seed)
    pos = rng.uniform(-half, half, (n, 3))
    vel = np.zeros((n, 3))
    mass = np.full(n, 1.0 / max(n, 1))
    return _pack(pos, vel, mass)


def random_cloud(n: int, seed: int, kind: str = "gauss"):
    """Small irregular clouds for edge-case tests (random masses in [0.5,1.5]/n).

    kind: "gauss" (normal), "planar" (z = 0), "clustered" (a few tight blobs),
    "line" (points on the x axis).
    """
    rng = _rng(seed)
    n = int(n)
    if kind == "gauss":
        pos = rng.normal(0.0, 1.0, (n, 3))
    elif kind == "planar":
        pos = np.concatenate([rng.uniform(-1, 1, (n, 2)), np.zeros((n, 1))], axis=1)
    elif kind == "clustered":
        k = max(1, n // 16)
        centres = rng.uniform(-1, 1, (k, 3))
        which = rng.integers(0, k, n)
        pos = centres[which] + rng.normal(0.0, 1e-4, (n, 3))
    elif kind == "line":
        pos = np.zeros((n, 3))
        pos[:, 0] = rng.uniform(-1, 1, n)
    else:
        raise ValueError(kind)
    vel = rng.normal(0.0, 0.1, (n, 3))
    mass = rng.uniform(0.5, 1.5, n) / max(n, 1)
    return _pack(pos, vel, mass)


def kepler_pair(m1: float = 0.6, m2: float = 0.4, a: float = 1.0, e: float = 0.5):
    """Two bodies at pericentre of a bound Kepler orbit (G = 1), COM at rest.

    Relative separation r_p = a (1 - e); relative speed from vis-viva
    v_p^2 = (m1 + m2) (2/r_p - 1/a).  Returned in FP32 layout; the FP64 values
    used to build them are returned too so closed-form tests can use them.
    """
    mt = m1 + m2
    rp = a * (1.0 - e)
    vp = math.sqrt(mt * (2.0 / rp - 1.0 / a))
    pos = np.array([[-m2 / mt * rp, 0.0, 0.0], [m1 / mt * rp, 0.0, 0.0]])
    vel = np.array([[0.0, -m2 / mt * vp, 0.0], [0.0, m1 / mt * vp, 0.0]])
    pm, v4 = _pack(pos, vel, np.array([m1, m2]))
    return pm, v4, dict(m1=m1, m2=m2, a=a, e=e, rp=rp, vp=vp,
                        period=2.0 * math.pi * math.sqrt(a ** 3 / mt))


@dataclass
class System:
    kind: str
    n: int
    seed: int
    theta: float
    eps: float
    pos_mass: np.ndarray = field(repr=False, default=None)
    vel: np.ndarray = field(repr=False, default=None)


def make_system(kind: str, n: int, seed: int):
    if kind == "plummer":
        return plummer(n, seed)
    if kind == "uniform":
        return uniform_cube(n, seed)
    raise ValueError(kind)


def forest_systems(n_systems: int = 512, n_min: int = 256, n_max: int = 65536,
                   seed: int = 4, theta: float = 0.5, eps: float = 0.01,
                   materialise: bool = True):
    """Many independent systems: N log-uniform in [n_min, n_max], even index
    Plummer, odd index uniform-cube cold collapse."""
    rng = _rng(seed)
    lo, hi = math.log(n_min), math.log(n_max)
    ns = np.rint(np.exp(rng.uniform(lo, hi, n_systems))).astype(np.int64)
    ns = np.clip(ns, n_min, n_max)
    seeds = rng.integers(1, 2 ** 31 - 1, n_systems)
    out = []
    for k in range(n_systems):
        kind = "plummer" if k % 2 == 0 else "uniform"
        s = System(kind, int(ns[k]), int(seeds[k]), theta, eps)
        if materialise:
            s.pos_mass, s.vel = make_system(kind, s.n, s.seed)
        out.append(s)
    return out


@dataclass
class Request:
    arrival_s: float
    kind: str
    n: int
    seed: int
    theta: float
    steps: int
    dt: float
    eps: float


def request_stream(rate_hz: float = 200.0, duration_s: float = 60.0,
                   n_min: int = 1024, n_max: int = 2097152, seed: int = 5,
                   theta_lo: float = 0.5, theta_hi: float = 0.8,
                   steps_lo: int = 10, steps_hi: int = 200, dt: float = 1e-3,
                   eps: float = 0.01):
    """Poisson request schedule (exponential inter-arrival times)."""
    rng = _rng(seed)
    t = 0.0
    out = []
    lo, hi = math.log(n_min), math.log(n_max)
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        kind = "plummer" if rng.uniform() < 0.5 else "uniform"
        n = int(min(n_max, max(n_min, round(math.exp(rng.uniform(lo, hi))))))
        out.append(Request(t, kind, n, int(rng.integers(1, 2 ** 31 - 1)),
                           float(rng.uniform(theta_lo, theta_hi)),
                           int(rng.integers(steps_lo, steps_hi + 1)), dt, eps))
    return out
