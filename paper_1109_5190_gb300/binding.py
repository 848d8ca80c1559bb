"""ctypes binding of ``libbh.so`` (declared in ``include/bh.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Functions keep the C names.  Arrays may be numpy arrays (host) or
torch CUDA tensors (device; ``BH_DEVICE_PTRS`` is added automatically) of
float32 with 4 values per particle.  A negative status raises ``BHError``.

The library must have been built (``__graft_entry__.build()`` or
``python -m paper_1109_5190_gb300._build``); importing this module without it
fails loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libbh.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libbh.so not built at {_LIB_PATH}; run __graft_entry__.build()")
lib = C.CDLL(_LIB_PATH)

BH_OK, BH_PENDING = 0, 1
BH_GROUP_LIST = 64  # bh_tuning.group: interaction-list walk
BH_GROUP_SIBLINGS = 65  # bh_tuning.group: one lane per particle over sibling-ordered nodes
BH_ERR_INVALID, BH_ERR_OOM, BH_ERR_BUDGET, BH_ERR_CAPACITY = -1, -2, -3, -4
BH_ERR_TIMEOUT, BH_ERR_CUDA, BH_ERR_STATE, BH_ERR_CANCELLED = -5, -6, -7, -8
BH_DEVICE_PTRS, BH_POTENTIAL, BH_NO_KAHAN, BH_OPEN_INSIDE, BH_QUADRUPOLE = 0x1, 0x2, 0x4, 0x8, 0x10
BH_OPEN_BMAX = 0x20
BH_MAX_DEPTH = 21
BH_NPHASE = 3


class BHError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class bh_params(C.Structure):
    _fields_ = [("G", C.c_double), ("eps", C.c_double), ("theta", C.c_double),
                ("max_depth", C.c_int), ("leaf_cap", C.c_int), ("flags", C.c_uint)]


class bh_node(C.Structure):
    _fields_ = [("prefix", C.c_uint64), ("first", C.c_uint32), ("count", C.c_uint32),
                ("level", C.c_uint8), ("childmask", C.c_uint8), ("pad", C.c_uint8 * 6)]


NODE_DTYPE = np.dtype([("prefix", "<u8"), ("first", "<u4"), ("count", "<u4"),
                       ("level", "u1"), ("childmask", "u1"), ("pad", "u1", (6,))])
assert NODE_DTYPE.itemsize == C.sizeof(bh_node) == 24


class bh_tuning(C.Structure):
    _fields_ = [("ppl", C.c_int), ("warps_per_block", C.c_int), ("blocks_per_sm", C.c_int),
                ("group", C.c_int), ("static_share", C.c_int)]


class bh_system_desc(C.Structure):
    _fields_ = [("n", C.c_int64), ("pos_mass", C.c_void_p), ("vel", C.c_void_p),
                ("G", C.c_double), ("eps", C.c_double), ("theta", C.c_double), ("dt", C.c_double)]


class bh_request(C.Structure):
    _fields_ = [("n", C.c_int64), ("pos_mass", C.c_void_p), ("vel", C.c_void_p),
                ("G", C.c_double), ("eps", C.c_double), ("theta", C.c_double), ("dt", C.c_double),
                ("nsteps", C.c_int), ("flags", C.c_uint)]


class bh_result(C.Structure):
    _fields_ = [("status", C.c_int), ("pad", C.c_int), ("pos_mass", C.c_void_p),
                ("vel", C.c_void_p), ("acc", C.c_void_p), ("submit_s", C.c_double),
                ("admit_s", C.c_double), ("done_s", C.c_double), ("steps_done", C.c_int64)]


class bh_server_stats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in (
        "submitted", "admitted", "completed", "rejected", "ticks", "particle_steps",
        "resident_systems", "peak_resident_systems", "resident_bytes", "peak_resident_bytes")] + \
        [("busy_s", C.c_double)]


P, I, U, I64, D, SZ = C.c_void_p, C.c_int, C.c_uint, C.c_int64, C.c_double, C.c_size_t
_SIGS = {
    "bh_last_error": ([], C.c_char_p),
    "bh_version": ([], C.c_char_p),
    "bh_params_default": ([P], I),
    "bh_create": ([P, P, I64, P, P, P, U], I),
    "bh_destroy": ([P], I),
    "bh_set_state": ([P, P, P, P, U], I),
    "bh_build_tree": ([P], I),
    "bh_get_tree": ([P, P, P, P, P, I64, P, P], I),
    "bh_compute_accel": ([P, P, U], I),
    "bh_step": ([P, I, D, I], I),
    "bh_get_state": ([P, P, P, P, U], I),
    "bh_diagnostics": ([P, P], I),
    "bh_interaction_count": ([P, P, P], I),
    "bh_walk_stats": ([P, P, P, P], I),
    "bh_set_tuning": ([P, P], I),
    "bh_get_tuning": ([P, P], I),
    "bh_autotune": ([P, P], I),
    "bh_profile_begin": ([P], I),
    "bh_profile_end": ([P, P, P, P], I),
    "bh_forest_create": ([P, I, P, P, U], I),
    "bh_forest_destroy": ([P], I),
    "bh_forest_compute_accel": ([P], I),
    "bh_forest_step": ([P, I, D, I], I),
    "bh_forest_get_state": ([P, I, P, P, P, U], I),
    "bh_forest_set_tuning": ([P, P], I),
    "bh_forest_autotune": ([P, P], I),
    "bh_forest_info": ([P, P, P], I),
    "bh_forest_profile_begin": ([P], I),
    "bh_forest_profile_end": ([P, P, P, P], I),
    "bh_server_create": ([P, SZ, I, P, U], I),
    "bh_submit": ([P, P, P], I),
    "bh_poll": ([P, C.c_uint64, P], I),
    "bh_wait": ([P, C.c_uint64, P, D], I),
    "bh_server_stats_get": ([P, P], I),
    "bh_server_now": ([P], D),
    "bh_server_destroy": ([P], I),
    "bh_partition_systems": ([I, P, I, P], I),
    "bh_morton_keys_noalloc": ([P, I64, P, P, P], I),
    "bh_micro_fma_peak": ([P, P], I),
    "bh_micro_l1_gather": ([P, P], I),
    "bh_micro_copy_bw": ([SZ, P, P], I),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _res


def bh_last_error() -> str:
    return lib.bh_last_error().decode()


def bh_version() -> str:
    return lib.bh_version().decode()


last_error = bh_last_error


def _check(rc: int) -> int:
    if rc < 0:
        raise BHError(rc, last_error())
    return rc


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _arr(x, n=None):
    """(pointer, device flag) of a float32 n x 4 array (numpy or torch CUDA)."""
    if x is None:
        return None, 0
    if _is_torch(x):
        import torch
        if x.dtype != torch.float32 or not x.is_contiguous():
            raise ValueError("torch tensors must be contiguous float32")
        if n is not None and x.numel() != 4 * n:
            raise ValueError("expected n x 4 values")
        return C.c_void_p(x.data_ptr()), (BH_DEVICE_PTRS if x.is_cuda else 0)
    if not (isinstance(x, np.ndarray) and x.dtype == np.float32 and x.flags.c_contiguous):
        raise ValueError("numpy arrays must be C-contiguous float32")
    if n is not None and x.size != 4 * n:
        raise ValueError("expected n x 4 values")
    return C.c_void_p(x.ctypes.data), 0


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def bh_params_default() -> bh_params:
    p = bh_params()
    _check(lib.bh_params_default(C.byref(p)))
    return p


def params(G=1.0, eps=0.01, theta=0.5, flags=0) -> bh_params:
    """bh_params_default() with G, eps, theta and flags set."""
    p = bh_params_default()
    p.G, p.eps, p.theta, p.flags = float(G), float(eps), float(theta), int(flags)
    return p


# ------------------------------------------------------------------ system

def bh_create(p: bh_params, pos_mass, vel=None, stream=None):
    n = (pos_mass.numel() if _is_torch(pos_mass) else pos_mass.size) // 4
    pp, f1 = _arr(pos_mass, n)
    vp, f2 = _arr(vel, n)
    if vel is not None and f1 != f2:
        raise ValueError("pos_mass and vel must both be host or both be device arrays")
    h = C.c_void_p()
    _check(lib.bh_create(C.byref(h), C.byref(p), n, pp, vp, _stream(stream), f1))
    return h


def bh_destroy(h):
    return _check(lib.bh_destroy(h))


def bh_set_state(h, pos_mass, vel=None, acc=None):
    pp, f1 = _arr(pos_mass)
    vp, _ = _arr(vel)
    ap, _ = _arr(acc)
    return _check(lib.bh_set_state(h, pp, vp, ap, f1))


def bh_build_tree(h):
    return _check(lib.bh_build_tree(h))


def bh_get_tree(h, n: int, node_cap: int | None = None):
    """Returns dict(keys, order, nodes (structured), com_m (M,4), cube (4,))."""
    nn = C.c_int64()
    _check(lib.bh_get_tree(h, None, None, None, None, 0, C.byref(nn), None))
    M = nn.value if node_cap is None else node_cap
    keys = np.zeros(n, np.uint64)
    order = np.zeros(n, np.uint32)
    nodes = np.zeros(M, NODE_DTYPE)
    com = np.zeros((M, 4), np.float32)
    cube = np.zeros(4, np.float32)
    _check(lib.bh_get_tree(h, keys.ctypes.data, order.ctypes.data, nodes.ctypes.data,
                           com.ctypes.data, M, C.byref(nn), cube.ctypes.data))
    M = nn.value
    return dict(keys=keys, order=order, nodes=nodes[:M], com_m=com[:M], cube=cube)


def bh_node_count(h) -> int:
    """Node count of the last built tree (bh_get_tree with no arrays)."""
    nn = C.c_int64()
    _check(lib.bh_get_tree(h, None, None, None, None, 0, C.byref(nn), None))
    return nn.value


def bh_compute_accel(h, acc_out=None):
    ap, f = _arr(acc_out)
    return _check(lib.bh_compute_accel(h, ap, f))


def bh_step(h, nsteps: int, dt: float, use_graph: bool = False):
    return _check(lib.bh_step(h, int(nsteps), float(dt), int(bool(use_graph))))


def bh_get_state(h, pos_mass=None, vel=None, acc=None):
    flags = 0
    ptrs = []
    for a in (pos_mass, vel, acc):
        p, f = _arr(a)
        ptrs.append(p)
        flags |= f
    return _check(lib.bh_get_state(h, *ptrs, flags))


def bh_diagnostics(h) -> np.ndarray:
    out = np.zeros(8, np.float64)
    _check(lib.bh_diagnostics(h, out.ctypes.data))
    return out


def bh_interaction_count(h, n: int):
    counts = np.zeros(n, np.uint32)
    tot = C.c_uint64()
    _check(lib.bh_interaction_count(h, counts.ctypes.data, C.byref(tot)))
    return counts, tot.value


def bh_walk_stats(h) -> dict:
    a, b, c = C.c_uint64(), C.c_uint64(), C.c_uint64()
    _check(lib.bh_walk_stats(h, C.byref(a), C.byref(b), C.byref(c)))
    return {"interactions": a.value, "warp_iterations": b.value, "slot_visits": c.value}


def bh_set_tuning(h, ppl=1, warps_per_block=16, blocks_per_sm=0, group=1, static_share=90):
    t = bh_tuning(ppl, warps_per_block, blocks_per_sm, group, static_share)
    return _check(lib.bh_set_tuning(h, C.byref(t)))


def bh_get_tuning(h) -> tuple:
    t = bh_tuning()
    _check(lib.bh_get_tuning(h, C.byref(t)))
    return (t.ppl, t.warps_per_block, t.blocks_per_sm, t.group, t.static_share)


def bh_autotune(h) -> tuple:
    t = bh_tuning()
    _check(lib.bh_autotune(h, C.byref(t)))
    return (t.ppl, t.warps_per_block, t.blocks_per_sm, t.group, t.static_share)


def bh_profile_begin(h):
    return _check(lib.bh_profile_begin(h))


def bh_profile_end(h):
    ph = np.zeros(BH_NPHASE, np.float64)
    steps = C.c_int64()
    launches = C.c_int64()
    _check(lib.bh_profile_end(h, ph.ctypes.data, C.byref(steps), C.byref(launches)))
    return ph, steps.value, launches.value


# ------------------------------------------------------------------ forest

def bh_forest_create(systems, stream=None, flags=0):
    """systems: list of dicts with pos_mass, vel, G, eps, theta, dt."""
    descs = (bh_system_desc * len(systems))()
    keep = []
    fl = 0
    for k, s in enumerate(systems):
        pm = s["pos_mass"]
        n = (pm.numel() if _is_torch(pm) else pm.size) // 4
        pp, f1 = _arr(pm, n)
        vp, _ = _arr(s.get("vel"), n)
        fl |= f1
        keep.append((pm, s.get("vel")))
        descs[k] = bh_system_desc(n, pp, vp, float(s.get("G", 1.0)), float(s.get("eps", 0.01)),
                                  float(s.get("theta", 0.5)), float(s.get("dt", 1e-3)))
    h = C.c_void_p()
    _check(lib.bh_forest_create(C.byref(h), len(systems), descs, _stream(stream), fl | int(flags)))
    return h


def bh_forest_destroy(h):
    return _check(lib.bh_forest_destroy(h))


def bh_forest_compute_accel(h):
    return _check(lib.bh_forest_compute_accel(h))


def bh_forest_step(h, nsteps: int, dt: float = 0.0, use_graph: bool = False):
    return _check(lib.bh_forest_step(h, int(nsteps), float(dt), int(bool(use_graph))))


def bh_forest_get_state(h, sys: int, pos_mass=None, vel=None, acc=None):
    flags = 0
    ptrs = []
    for a in (pos_mass, vel, acc):
        p, f = _arr(a)
        ptrs.append(p)
        flags |= f
    return _check(lib.bh_forest_get_state(h, int(sys), *ptrs, flags))


def bh_forest_set_tuning(h, ppl=1, warps_per_block=16, blocks_per_sm=0, group=1, static_share=0):
    t = bh_tuning(ppl, warps_per_block, blocks_per_sm, group, static_share)
    return _check(lib.bh_forest_set_tuning(h, C.byref(t)))


def bh_forest_autotune(h) -> tuple:
    t = bh_tuning()
    _check(lib.bh_forest_autotune(h, C.byref(t)))
    return (t.ppl, t.warps_per_block, t.blocks_per_sm, t.group, t.static_share)


def bh_forest_info(h):
    a, b = C.c_int64(), C.c_int64()
    _check(lib.bh_forest_info(h, C.byref(a), C.byref(b)))
    return a.value, b.value


def bh_forest_profile_begin(h):
    return _check(lib.bh_forest_profile_begin(h))


def bh_forest_profile_end(h):
    ph = np.zeros(BH_NPHASE, np.float64)
    steps = C.c_int64()
    launches = C.c_int64()
    _check(lib.bh_forest_profile_end(h, ph.ctypes.data, C.byref(steps), C.byref(launches)))
    return ph, steps.value, launches.value


# ------------------------------------------------------------------ server

def bh_server_create(hbm_budget: int, max_slots: int, stream=None, flags=0):
    h = C.c_void_p()
    _check(lib.bh_server_create(C.byref(h), C.c_size_t(int(hbm_budget)), int(max_slots),
                                _stream(stream), int(flags)))
    return h


def bh_submit(h, pos_mass, vel=None, G=1.0, eps=0.01, theta=0.5, dt=1e-3, nsteps=0, flags=0):
    n = pos_mass.size // 4
    pp, f = _arr(pos_mass, n)
    vp, _ = _arr(vel, n)
    if f:
        raise ValueError("requests take host arrays")
    r = bh_request(n, pp, vp, float(G), float(eps), float(theta), float(dt), int(nsteps), int(flags))
    t = C.c_uint64()
    _check(lib.bh_submit(h, C.byref(r), C.byref(t)))
    return t.value


def _result(n, want):
    out = {}
    res = bh_result()
    for k in ("pos_mass", "vel", "acc"):
        if want:
            out[k] = np.zeros((n, 4), np.float32)
            setattr(res, k, out[k].ctypes.data)
    return res, out


def bh_poll(h, ticket: int, n: int = 0):
    """None while pending; dict(status, arrays..., times) once done."""
    res, out = _result(n, n > 0)
    rc = lib.bh_poll(h, C.c_uint64(ticket), C.byref(res))
    if rc == BH_PENDING:
        return None
    _check(rc)
    out.update(status=res.status, submit_s=res.submit_s, admit_s=res.admit_s, done_s=res.done_s,
               steps_done=res.steps_done)
    return out


def bh_wait(h, ticket: int, n: int = 0, timeout_s: float = 60.0):
    res, out = _result(n, n > 0)
    _check(lib.bh_wait(h, C.c_uint64(ticket), C.byref(res), float(timeout_s)))
    out.update(status=res.status, submit_s=res.submit_s, admit_s=res.admit_s, done_s=res.done_s,
               steps_done=res.steps_done)
    return out


def bh_server_stats_get(h) -> dict:
    st = bh_server_stats()
    _check(lib.bh_server_stats_get(h, C.byref(st)))
    return {k: getattr(st, k) for k, _ in bh_server_stats._fields_}


def bh_server_now(h) -> float:
    return lib.bh_server_now(h)


def bh_server_destroy(h):
    return _check(lib.bh_server_destroy(h))


# ---------------------------------------------------------------- sharding

def bh_partition_systems(sizes, world: int) -> np.ndarray:
    """Rank of each system (bh_partition_systems) for `world` ranks."""
    n = np.ascontiguousarray(np.asarray(sizes, dtype=np.int64))
    out = np.zeros(n.size, np.int32)
    _check(lib.bh_partition_systems(int(n.size), n.ctypes.data if n.size else None, int(world),
                                    out.ctypes.data if n.size else None))
    return out


# ------------------------------------------------- allocation-free Morton keys

BH_NOALLOC_MAX_N = 16777216
BH_NOALLOC_BAD_KEY = 0xffffffffffffffff


def bh_morton_keys_noalloc(pos_mass, keys, cube=None, stream=None):
    """Keys of device pos_mass (n x 4 float32) into device keys (n int64 /
    uint64 tensor) and cube (4 float32 or None); enqueued on `stream`, no
    allocation.  For callers that cannot allocate device memory.  Every
    tensor must be a contiguous CUDA tensor of the stated type and size."""
    import torch
    for name, t in (("pos_mass", pos_mass), ("keys", keys), ("cube", cube)):
        if t is None and name == "cube":
            continue
        if not (_is_torch(t) and t.is_cuda and t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous CUDA tensor")
    if pos_mass.dtype != torch.float32 or pos_mass.dim() != 2 or pos_mass.shape[1] != 4:
        raise ValueError("pos_mass must be float32 of shape (n, 4)")
    n = pos_mass.shape[0]
    if keys.dtype not in (torch.int64, getattr(torch, "uint64", torch.int64)) or keys.numel() != n:
        raise ValueError("keys must hold n 64-bit integers")
    if cube is not None and (cube.dtype != torch.float32 or cube.numel() < 4):
        raise ValueError("cube must be float32 with at least 4 values")
    devs = {t.device for t in (pos_mass, keys, cube) if t is not None}
    if len(devs) != 1:
        raise ValueError("pos_mass, keys and cube must be on one device")
    cp = C.c_void_p(cube.data_ptr()) if cube is not None else None
    with torch.cuda.device(pos_mass.device):
        return _check(lib.bh_morton_keys_noalloc(C.c_void_p(pos_mass.data_ptr()), n,
                                                 C.c_void_p(keys.data_ptr()), cp,
                                                 _stream(stream)))


# ---------------------------------------------------------- micro-benchmarks

def bh_micro_fma_peak(stream=None) -> float:
    g = C.c_double()
    _check(lib.bh_micro_fma_peak(C.byref(g), _stream(stream)))
    return g.value


def bh_micro_l1_gather(stream=None) -> float:
    """G sectors/s of scattered 32-byte L1 loads (the walk's node loads)."""
    g = C.c_double()
    _check(lib.bh_micro_l1_gather(C.byref(g), _stream(stream)))
    return g.value


def bh_micro_copy_bw(nbytes: int, stream=None) -> float:
    g = C.c_double()
    _check(lib.bh_micro_copy_bw(C.c_size_t(int(nbytes)), C.byref(g), _stream(stream)))
    return g.value
