"""The C-ABI library loads and exports every function that include/*.h
declares (no GPU work is done here), plus host-side argument checks that fail
before touching the device."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    path = __graft_entry__._builder().build()
    return ctypes.CDLL(path)


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(bh_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("bh_create", "bh_build_tree", "bh_compute_accel", "bh_step",
                     "bh_submit", "bh_poll", "bh_forest_create", "bh_forest_step",
                     "bh_server_create", "bh_get_tree", "bh_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_symbol(lib):
    from paper_1109_5190_gb300 import binding
    missing = [n for n in declared_functions() if n not in binding._SIGS]
    assert not missing, missing
    # and offers a Python function of the same name for each
    unnamed = [n for n in declared_functions() if not callable(getattr(binding, n, None))]
    assert not unnamed, unnamed


def test_binding_constants_match_the_header():
    # every #define of include/bh.h with an integer value has the same value
    # in the binding (status codes, flags, limits)
    from paper_1109_5190_gb300 import binding as B
    text = open(os.path.join(ROOT, "include", "bh.h")).read()
    found = 0
    for m in re.finditer(r"^#define\s+(BH_[A-Z0-9_]+)\s+\(?(-?(?:0x[0-9a-fA-F]+|\d+))u?\)?",
                         text, flags=re.M):
        name, val = m.group(1), int(m.group(2), 0)
        assert getattr(B, name, None) == val, name
        found += 1
    assert found >= 20 and B.BH_OPEN_BMAX == 0x20


def test_host_side_argument_errors(lib):
    from paper_1109_5190_gb300 import binding as B
    import numpy as np
    p = B.params()
    assert B.lib.bh_params_default(None) == B.BH_ERR_INVALID
    # invalid parameters are rejected before any device call
    bad = B.params(G=-1.0)
    h = ctypes.c_void_p()
    pm = np.zeros((4, 4), np.float32)
    pm[:, 3] = 1.0
    assert B.lib.bh_create(ctypes.byref(h), ctypes.byref(bad), 4, pm.ctypes.data, None, None, 0) \
        == B.BH_ERR_INVALID
    assert "G" in B.last_error()
    bad = B.params(theta=-0.1)
    assert B.lib.bh_create(ctypes.byref(h), ctypes.byref(bad), 4, pm.ctypes.data, None, None, 0) \
        == B.BH_ERR_INVALID
    assert B.lib.bh_create(ctypes.byref(h), ctypes.byref(p), 0, pm.ctypes.data, None, None, 0) \
        == B.BH_ERR_INVALID
    p.max_depth = 20
    assert B.lib.bh_create(ctypes.byref(h), ctypes.byref(p), 4, pm.ctypes.data, None, None, 0) \
        == B.BH_ERR_INVALID
    p = B.params(flags=0x40)  # no such flag
    assert B.lib.bh_create(ctypes.byref(h), ctypes.byref(p), 4, pm.ctypes.data, None, None, 0) \
        == B.BH_ERR_INVALID
    # quadrupoles need Kahan sums: rejected before any device work, for a
    # system, a forest and a server alike
    p = B.params(flags=B.BH_QUADRUPOLE | B.BH_NO_KAHAN)
    assert B.lib.bh_create(ctypes.byref(h), ctypes.byref(p), 4, pm.ctypes.data, None, None, 0) \
        == B.BH_ERR_INVALID
    assert "Kahan" in B.last_error()
    d = (B.bh_system_desc * 1)()
    d[0].n, d[0].pos_mass, d[0].G, d[0].eps, d[0].theta, d[0].dt = 4, pm.ctypes.data, 1.0, 0.01, 0.5, 1e-3
    for fl in (B.BH_QUADRUPOLE | B.BH_NO_KAHAN, 0x40):
        assert B.lib.bh_forest_create(ctypes.byref(h), 1, d, None, fl) == B.BH_ERR_INVALID
        assert B.lib.bh_server_create(ctypes.byref(h), 1 << 30, 2, None, fl) == B.BH_ERR_INVALID
    assert B.lib.bh_server_create(ctypes.byref(h), 1 << 10, 2, None, 0) == B.BH_ERR_INVALID  # budget
    assert B.lib.bh_step(None, 1, 1e-3, 0) == B.BH_ERR_INVALID
    assert B.lib.bh_poll(None, 1, None) == B.BH_ERR_INVALID
    assert B.lib.bh_version().decode().startswith("bh-gb300")


def test_oracle_and_library_share_no_code():
    # the oracle is plain C in oracle/; the library's sources never include or
    # name it, and the oracle never includes the library's headers
    for src in glob.glob(os.path.join(ROOT, "paper_1109_5190_gb300", "**", "*"), recursive=True):
        if os.path.isfile(src) and src.endswith((".cu", ".cuh", ".h", ".py", ".cpp")):
            text = open(src, errors="ignore").read()
            assert "import oracle" not in text and "bh_oracle" not in text, src
    otext = open(os.path.join(ROOT, "oracle", "bh_oracle.c")).read()
    assert "#include \"bh" not in otext and "bh_internal" not in otext
