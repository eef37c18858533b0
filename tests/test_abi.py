"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/lp.h declares (no compute call: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "lp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lp_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_entry_points():
    syms = declared_symbols()
    for s in ("lp_create", "lp_destroy", "lp_build_neighbors", "lp_gfd_derivs", "lp_step"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    from paper_2206_11998_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    from paper_2206_11998_gb300 import lp
    assert set(declared_symbols()) <= set(lp.EXPORTED)


def test_host_side_argument_errors_without_gpu():
    # lp_create validates its configuration before touching the device
    from paper_2206_11998_gb300 import build, lp
    build.build()
    L = lp.lib()
    h = ctypes.c_void_p()
    bad = lp.make_config(4, 100)                    # dim out of range
    assert L.lp_create(ctypes.byref(bad), ctypes.byref(h)) == lp.ERR_ARG
    bad = lp.make_config(3, 100, k_max=81)          # above the compiled capacity
    assert L.lp_create(ctypes.byref(bad), ctypes.byref(h)) == lp.ERR_ARG
    bad = lp.make_config(2, 100, periodic=(1, 1, 0), box_hi=(1.0, 2.0, 1.0))   # non-cubic periodic box
    assert L.lp_create(ctypes.byref(bad), ctypes.byref(h)) == lp.ERR_ARG
    bad = lp.make_config(2, 100, periodic=(1, 0, 0))   # periodic on some axes only
    assert L.lp_create(ctypes.byref(bad), ctypes.byref(h)) == lp.ERR_ARG
    bad = lp.make_config(3, 100, radius_mode=lp.RADIUS_KSIDE)   # k-per-side is 1D only
    assert L.lp_create(ctypes.byref(bad), ctypes.byref(h)) == lp.ERR_ARG
    assert L.lp_create(None, ctypes.byref(h)) == lp.ERR_ARG
    assert L.lp_set_schedule(None, lp.SCHED_SPLIT) == lp.ERR_ARG
    assert L.lp_autotune(None, None, None, 1, 0.0, 0.4, 1, None, None) == lp.ERR_ARG
    assert L.lp_step_host(None, None, 0.0, 0.4, None, None, None) == lp.ERR_ARG
    assert L.lp_destroy(None) == lp.OK
    assert L.lp_status_string(lp.ERR_CAPACITY).decode().startswith("particle count")


def test_noalloc_binding_checks_its_buffers():
    """The binding refuses buffers the entry point would overrun or misread
    (wrong dtype, host memory, too short) before calling the library."""
    torch = pytest.importorskip("torch")
    from paper_2206_11998_gb300 import lp
    x = [torch.zeros(10, dtype=torch.float64)]
    keys = torch.zeros(10, dtype=torch.int64)
    perm = torch.zeros(10, dtype=torch.int32)
    with pytest.raises(ValueError):
        lp.sort_keys_noalloc(x, keys, perm)                      # host tensors
    with pytest.raises(ValueError):
        lp.sort_keys_noalloc([torch.zeros(10, dtype=torch.float32)], keys, perm)
    with pytest.raises(ValueError):
        lp.sort_keys_noalloc([], keys, perm)
