"""The allocation-free Morton-key entry point.

bh_morton_keys_noalloc serves callers that cannot allocate device memory (see
its comment in include/bh.h): its scratch is a static device array, so it
calls no allocator.  Here it is checked, through the C ABI, against the keys
and key cube that the regular tree build computes for the same particles and
against the FP64 oracle's keys and cube, on calls in a row with different
inputs (a call must not see the previous call's leftovers), up to its largest
size.  Keys are integers: equality is exact.  Arguments a kernel could not use
in place are rejected on the host before any launch; the tests below that
pass such arguments never reach a kernel.  This file is collected last so
that a failure here cannot hide the other tests.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1109_5190_gb300 import binding as B  # noqa: E402


def regular_keys(pm):
    """Keys (input order) and cube from the regular build (bh_build_tree)."""
    h = B.bh_create(B.params(), pm)
    try:
        B.bh_build_tree(h)
        t = B.bh_get_tree(h, len(pm))
    finally:
        B.bh_destroy(h)
    keys = np.zeros(len(pm), np.uint64)
    keys[t["order"].astype(np.int64)] = t["keys"]
    return keys, t["cube"]


def oracle_keys(pm):
    lo, side = oracle.cube(pm)
    return oracle.keys(pm), np.array([lo[0], lo[1], lo[2], side], np.float32)


def noalloc_keys(pm, stream):
    d_pm = torch.from_numpy(pm).cuda()
    d_keys = torch.zeros(len(pm), dtype=torch.int64, device="cuda")
    d_cube = torch.zeros(4, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    B.bh_morton_keys_noalloc(d_pm, d_keys, d_cube, stream)
    stream.synchronize()
    return d_keys.cpu().numpy().view(np.uint64), d_cube.cpu().numpy()


def test_noalloc_keys_match_the_tree_build_twice_in_a_row():
    stream = torch.cuda.Stream()
    # a large Plummer sphere, then a small uniform cube with another extent:
    # the second call must overwrite every scratch entry it uses
    inputs = [synth.plummer(300_001, 31)[0], synth.uniform_cube(5_000, 32, half=3.0)[0]]
    for pm in inputs:
        want_keys, want_cube = regular_keys(pm)
        got_keys, got_cube = noalloc_keys(pm, stream)
        assert np.array_equal(got_cube, want_cube)
        assert np.array_equal(got_keys, want_keys)
        o_keys, o_cube = oracle_keys(pm)
        assert np.array_equal(got_cube, o_cube)
        assert np.array_equal(got_keys, o_keys)


def test_noalloc_keys_at_the_largest_size_match_the_oracle():
    # n = BH_NOALLOC_MAX_N: every chunk slot of the static scratch is used and
    # the key kernel's grid (capped at 65,535 blocks) strides over the input
    stream = torch.cuda.Stream()
    n = B.BH_NOALLOC_MAX_N
    pm = synth.uniform_cube(n, 33, half=1.5)[0]
    pm[::7, :3] += np.float32(0.25)  # an uneven cloud, so every axis matters
    want_keys, want_cube = oracle_keys(pm)
    got_keys, got_cube = noalloc_keys(pm, stream)
    assert np.array_equal(got_cube, want_cube)
    assert np.array_equal(got_keys, want_keys)
    # and a small call right after it: the big call's leftovers are not read
    pm2 = synth.plummer(4_097, 34)[0]
    want2, cube2 = oracle_keys(pm2)
    got2, gcube2 = noalloc_keys(pm2, stream)
    assert np.array_equal(gcube2, cube2)
    assert np.array_equal(got2, want2)


def test_noalloc_marks_non_finite_input_then_recovers():
    stream = torch.cuda.Stream()
    for bad in (np.nan, np.inf, -np.inf):
        pm = synth.uniform_cube(10_000, 35)[0]
        pm[5_003, 1] = bad
        got_keys, got_cube = noalloc_keys(pm, stream)
        assert np.all(got_keys == np.uint64(B.BH_NOALLOC_BAD_KEY))
        assert np.all(np.isnan(got_cube))
    # a finite input after a marked one gets its true keys again
    pm = synth.uniform_cube(10_000, 36)[0]
    want_keys, want_cube = oracle_keys(pm)
    got_keys, got_cube = noalloc_keys(pm, stream)
    assert np.array_equal(got_cube, want_cube)
    assert np.array_equal(got_keys, want_keys)


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    pm = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    keys = torch.zeros(4, dtype=torch.int64, device="cuda")
    rc = B.lib.bh_morton_keys_noalloc(C.c_void_p(pm.data_ptr()), B.BH_NOALLOC_MAX_N + 1,
                                      C.c_void_p(keys.data_ptr()), None, None)
    assert rc == B.BH_ERR_INVALID
    assert "static scratch" in B.last_error()
    rc = B.lib.bh_morton_keys_noalloc(C.c_void_p(pm.data_ptr()), 0,
                                      C.c_void_p(keys.data_ptr()), None, None)
    assert rc == B.BH_ERR_INVALID


def test_noalloc_rejects_host_and_misaligned_pointers_before_any_launch():
    n = 64
    d_pm = torch.ones((n + 1, 4), dtype=torch.float32, device="cuda")
    d_keys = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    d_cube = torch.zeros(8, dtype=torch.float32, device="cuda")
    h_pm = np.ones((n, 4), np.float32)
    p_pm = torch.ones((n, 4), dtype=torch.float32).pin_memory()
    h_keys = np.zeros(n, np.uint64)
    dev = lambda t, off=0: C.c_void_p(t.data_ptr() + off)  # noqa: E731
    host = lambda a: C.c_void_p(a.ctypes.data)  # noqa: E731
    cases = [
        (host(h_pm), dev(d_keys), dev(d_cube), "pos_mass"),        # pageable host
        (dev(p_pm), dev(d_keys), dev(d_cube), "pos_mass"),         # pinned host
        (dev(d_pm), host(h_keys), dev(d_cube), "keys"),            # host keys
        (dev(d_pm), dev(d_keys), host(h_pm), "cube"),              # host cube
        (dev(d_pm, 4), dev(d_keys), dev(d_cube), "pos_mass"),      # not 16-byte aligned
        (dev(d_pm), dev(d_keys, 4), dev(d_cube), "keys"),          # not 8-byte aligned
        (dev(d_pm), dev(d_keys), dev(d_cube, 2), "cube"),          # not 4-byte aligned
    ]
    for pm_p, k_p, c_p, what in cases:
        rc = B.lib.bh_morton_keys_noalloc(pm_p, n, k_p, c_p, None)
        assert rc == B.BH_ERR_INVALID, what
        assert what in B.last_error()
    # nothing was written: the device outputs still hold their initial values
    torch.cuda.synchronize()
    assert int(d_keys.abs().sum()) == 0 and float(d_cube.abs().sum()) == 0.0


def test_noalloc_binding_rejects_wrong_tensors():
    n = 32
    good_pm = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    good_keys = torch.zeros(n, dtype=torch.int64, device="cuda")
    bad = [
        (good_pm.double(), good_keys, None),                            # float64 input
        (good_pm.half(), good_keys, None),                              # half input
        (torch.zeros((4, n), device="cuda").t(), good_keys, None),      # not contiguous
        (good_pm.reshape(-1), good_keys, None),                         # not (n, 4)
        (good_pm.cpu(), good_keys, None),                               # host tensor
        (good_pm, good_keys[: n - 1], None),                            # too few keys
        (good_pm, good_keys.int(), None),                               # 32-bit keys
        (good_pm, good_keys, torch.zeros(3, device="cuda")),            # cube too small
        (good_pm, good_keys, torch.zeros(4, dtype=torch.float64, device="cuda")),
    ]
    for pm, keys, cube in bad:
        with pytest.raises(ValueError):
            B.bh_morton_keys_noalloc(pm, keys, cube)
