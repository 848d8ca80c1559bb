"""FP64 CPU oracle for the Barnes-Hut hot path (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package.  It shares no code with the GPU library and never
imports it.  The arithmetic lives in ``bh_oracle.c`` (plain C, FP64); this
module only marshals numpy arrays through ctypes.

Every function follows the paper (Dekate et al., arXiv:1109.5190) as read in
``bh_oracle.c``: the octree of Section I (one particle per leaf), the centre
of mass per cube (Section I, Fig. 2), the opening criterion of Section III
(Fig. 1), and the readings listed at the top of ``bh_oracle.c`` for what the
paper leaves unstated (force law, keys, integrator).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bh_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp"]


def build(force: bool = False) -> str:
    """Compile ``bh_oracle.c`` into ``liboracle.so`` (gcc, no CUDA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        L = C.CDLL(_LIB)
        P = C.c_void_p
        i64, dbl, i32 = C.c_int64, C.c_double, C.c_int
        L.oracle_nsum.argtypes = [i64, P]
        L.oracle_nsum.restype = dbl
        L.oracle_cube.argtypes = [i64, P, P, P]
        L.oracle_keys.argtypes = [i64, P, P, P, P]
        L.oracle_tree_build.argtypes = [i64, P]
        L.oracle_tree_build.restype = P
        L.oracle_tree_free.argtypes = [P]
        L.oracle_tree_nnodes.argtypes = [P]
        L.oracle_tree_nnodes.restype = i64
        L.oracle_tree_cube.argtypes = [P, P, P]
        L.oracle_tree_export.argtypes = [P, P, P, P, P, P, P, P]
        L.oracle_tree_order.argtypes = [P, P, P]
        L.oracle_accel.argtypes = [P, dbl, dbl, dbl, i64, P, P, P, P, i32, i32]
        L.oracle_accel.restype = i32
        L.oracle_direct.argtypes = [i64, P, dbl, dbl, i64, P, P, P, i32]
        L.oracle_direct.restype = i32
        L.oracle_leapfrog.argtypes = [i64, P, P, P, i32, dbl, dbl, dbl, i32, dbl, i32]
        L.oracle_leapfrog.restype = i32
        L.oracle_diagnostics.argtypes = [i64, P, P, P, P]
        _lib = L
        return L


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _pm64(pos_mass) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(pos_mass, dtype=np.float64).reshape(-1, 4))
    return a


def nsum(x) -> float:
    """Neumaier-compensated sum of a float64 vector."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    return _load().oracle_nsum(x.size, _ptr(x))


def cube(pos_mass):
    """(lo[3] float32, side float32) of the key rule's bounding cube."""
    pm = _pm64(pos_mass)
    lo = np.zeros(3, np.float32)
    side = np.zeros(1, np.float32)
    _load().oracle_cube(pm.shape[0], _ptr(pm), _ptr(lo), _ptr(side))
    return lo, side[0]


def keys(pos_mass) -> np.ndarray:
    """63-bit Morton keys (uint64) of each input particle."""
    pm = _pm64(pos_mass)
    k = np.zeros(pm.shape[0], np.uint64)
    _load().oracle_keys(pm.shape[0], _ptr(pm), _ptr(k), None, None)
    return k


class Tree:
    """Recursive-insertion octree of one system (FP64 masses and centres)."""

    def __init__(self, pos_mass):
        self.pm = _pm64(pos_mass)
        L = _load()
        self._h = L.oracle_tree_build(self.pm.shape[0], _ptr(self.pm))
        if not self._h:
            raise ValueError("oracle tree build failed (empty input, non-positive mass or OOM)")
        self.n = self.pm.shape[0]
        self.m = L.oracle_tree_nnodes(self._h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _load().oracle_tree_free(h)
            self._h = None

    def cube(self):
        lo = np.zeros(3, np.float32)
        side = np.zeros(1, np.float32)
        _load().oracle_tree_cube(self._h, _ptr(lo), _ptr(side))
        return lo, side[0]

    def nodes(self) -> dict:
        """Canonical node list (depth-first pre-order, octant order)."""
        M = self.m
        out = dict(level=np.zeros(M, np.int32), prefix=np.zeros(M, np.uint64),
                   first=np.zeros(M, np.int64), count=np.zeros(M, np.int64),
                   childmask=np.zeros(M, np.int32), mass=np.zeros(M, np.float64),
                   com=np.zeros((M, 3), np.float64))
        _load().oracle_tree_export(self._h, *(_ptr(out[k]) for k in
                                   ("level", "prefix", "first", "count", "childmask", "mass", "com")))
        return out

    def order(self):
        """(order, keys): order[k] = input index of the k-th particle in
        canonical order; keys[i] = key of input particle i."""
        o = np.zeros(self.n, np.int64)
        k = np.zeros(self.n, np.uint64)
        _load().oracle_tree_order(self._h, _ptr(o), _ptr(k))
        return o, k

    def accel(self, theta: float, eps: float, G: float = 1.0, targets=None,
              nthreads: int = 0, open_inside: bool = False, quadrupole: bool = False,
              bmax: bool = False):
        """(acc (nt,3), pot (nt,), count (nt,)) for the target input indices.
        open_inside: never accept a cell that contains the particle;
        quadrupole: accepted cells add their second-order term;
        bmax: the opening test uses b_max (centre of mass to the cell's
        farthest corner) for the cell's size instead of its side."""
        if targets is None:
            nt, tp = self.n, None
        else:
            tp = np.ascontiguousarray(np.asarray(targets, dtype=np.int64))
            nt = tp.size
        acc = np.zeros((nt, 3), np.float64)
        pot = np.zeros(nt, np.float64)
        cnt = np.zeros(nt, np.int64)
        _load().oracle_accel(self._h, G, eps, theta, nt, _ptr(tp), _ptr(acc), _ptr(pot),
                             _ptr(cnt), int(nthreads),
                             int(bool(open_inside)) | (2 if quadrupole else 0)
                             | (4 if bmax else 0))
        return acc, pot, cnt


def direct(pos_mass, eps: float, G: float = 1.0, targets=None, nthreads: int = 0):
    """Direct O(n^2) sum: (acc (nt,3), pot (nt,))."""
    pm = _pm64(pos_mass)
    if targets is None:
        nt, tp = pm.shape[0], None
    else:
        tp = np.ascontiguousarray(np.asarray(targets, dtype=np.int64))
        nt = tp.size
    acc = np.zeros((nt, 3), np.float64)
    pot = np.zeros(nt, np.float64)
    _load().oracle_direct(pm.shape[0], _ptr(pm), G, eps, nt, _ptr(tp), _ptr(acc), _ptr(pot),
                          int(nthreads))
    return acc, pot


def accel(pos_mass, theta: float, eps: float, G: float = 1.0, targets=None, nthreads=0):
    return Tree(pos_mass).accel(theta, eps, G, targets, nthreads)


def leapfrog(pos_mass, vel, nsteps: int, dt: float, theta: float, eps: float,
             G: float = 1.0, acc=None, nthreads: int = 0):
    """FP64 KDK leapfrog; returns (pos_mass (n,4) f64, vel (n,3) f64, acc (n,3))."""
    pm = _pm64(pos_mass).copy()
    v = np.ascontiguousarray(np.asarray(vel, dtype=np.float64)[:, :3]).copy()
    have = acc is not None
    a = np.ascontiguousarray(np.asarray(acc, dtype=np.float64)).copy() if have else \
        np.zeros((pm.shape[0], 3), np.float64)
    rc = _load().oracle_leapfrog(pm.shape[0], _ptr(pm), _ptr(v), _ptr(a), int(have), G, eps,
                                 theta, int(nsteps), float(dt), int(nthreads))
    if rc:
        raise RuntimeError("oracle leapfrog failed")
    return pm, v, a


def diagnostics(pos_mass, vel, phi=None) -> np.ndarray:
    """[KE, PE, Px, Py, Pz, COMx, COMy, COMz] in FP64."""
    pm = _pm64(pos_mass)
    v = np.ascontiguousarray(np.asarray(vel, dtype=np.float64)[:, :3])
    ph = None if phi is None else np.ascontiguousarray(np.asarray(phi, dtype=np.float64))
    out = np.zeros(8, np.float64)
    _load().oracle_diagnostics(pm.shape[0], _ptr(pm), _ptr(v), _ptr(ph), _ptr(out))
    return out
