"""The allocation-free Morton-key entry point.

bh_morton_keys_noalloc serves callers that cannot allocate device memory (see
its comment in include/bh.h): its scratch is a static device array, so it
calls no allocator.  Here it is checked, through the C ABI, against the keys
and key cube that the regular tree build computes for the same particles, on
two calls in a row with different inputs (the second call must not see the
first call's leftovers).  Keys are integers: equality is exact.  This file
is collected last so that a failure here cannot hide the other tests.
"""
import numpy as np
import pytest

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


def noalloc_keys(pm, stream):
    d_pm = torch.from_numpy(pm).cuda()
    d_keys = torch.zeros(len(pm), dtype=torch.int64, device="cuda")
    d_cube = torch.zeros(4, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
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


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    pm = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    keys = torch.zeros(4, dtype=torch.int64, device="cuda")
    rc = B.lib.bh_morton_keys_noalloc(B.C.c_void_p(pm.data_ptr()), B.BH_NOALLOC_MAX_N + 1,
                                      B.C.c_void_p(keys.data_ptr()), None, None)
    assert rc == B.BH_ERR_INVALID
    assert "static scratch" in B.last_error()
    rc = B.lib.bh_morton_keys_noalloc(B.C.c_void_p(pm.data_ptr()), 0,
                                      B.C.c_void_p(keys.data_ptr()), None, None)
    assert rc == B.BH_ERR_INVALID
