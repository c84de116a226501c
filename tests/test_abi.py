"""The C-ABI library builds for sm_103a, loads, and exports every function the
public header declares (no device calls here)."""
import ctypes
import os
import re

import pytest

import paper_2408_10743_gb300 as dist
from paper_2408_10743_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dist.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\*?\s*(dist_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("dist_init", "dist_solve", "dist_solve_bounded", "dist_free", "dist_set_exclude",
                 "dist_strerror", "dist_intpeak"):
        assert must in names


def test_library_exports_every_declared_symbol():
    L = ctypes.CDLL(dist.library_path() if os.path.exists(dist.library_path()) else dist.lib()._name)
    for name in declared_functions():
        assert hasattr(L, name), name
    # the binding wraps every declared function with the same name
    assert set(declared_functions()) <= set(binding.SIGNATURES)


def test_library_is_in_tree_and_built_for_sm103a():
    path = dist.library_path()
    dist.lib()
    assert os.path.exists(path)
    assert os.path.dirname(path).startswith(ROOT)
    log = open(os.path.join(os.path.dirname(path), "_build", "compile.log")).read()
    assert "arch=compute_103a,code=sm_103a" in log


def test_strerror_and_version():
    assert "sm_103a" in dist.dist_version()
    assert dist.dist_strerror(-6).startswith("no nonzero")
    assert dist.dist_strerror(12345) == "unknown error"


def test_invalid_arguments_rejected_without_device():
    import numpy as np
    with pytest.raises(dist.DistError) as e:
        dist.dist_plan_info_get(np.array([[2, 0]], dtype=np.uint8))
    assert e.value.code == -1
    with pytest.raises(dist.DistError) as e:
        dist.dist_plan_info_get(np.zeros((2, 6), dtype=np.uint8))
    assert e.value.code == -6


def test_tuning_get_set_clamps():
    saved = dist.dist_get_tuning()
    try:
        dist.dist_set_tuning(1000, 2, 30)
        t = dist.dist_get_tuning()
        assert t["chunks_per_warp"] == 256 and t["lane_cap_log2"] == 8
        assert t["lane_floor_log2"] == 8  # never above the cap
        dist.dist_set_tuning(0, 0, 0)  # zero keeps the current values
        assert dist.dist_get_tuning() == t
        dist.dist_set_tuning(3, 20, 12)
        assert dist.dist_get_tuning() == {"chunks_per_warp": 3, "lane_cap_log2": 20,
                                          "lane_floor_log2": 12}
    finally:
        dist.dist_set_tuning(saved["chunks_per_warp"], saved["lane_cap_log2"],
                             saved["lane_floor_log2"])


def test_init_many_rejects_bad_arguments_without_device():
    """dist_init_many checks its arguments before it touches a device: a
    negative count or a missing array is DIST_EINVAL, and count 0 is accepted
    with nothing to do."""
    L = dist.lib()
    n = (ctypes.c_int * 1)(4)
    K = (ctypes.c_int * 1)(2)
    f = (ctypes.c_int * 1)(dist.DIST_F2)
    st = (ctypes.c_int * 1)()
    out = (ctypes.c_void_p * 1)()
    g = (ctypes.c_uint8 * 16)()
    gens = (ctypes.POINTER(ctypes.c_uint8) * 1)(ctypes.cast(g, ctypes.POINTER(ctypes.c_uint8)))
    assert L.dist_init_many(out, -1, gens, n, K, f, st) == -1
    assert L.dist_init_many(out, 1, None, n, K, f, st) == -1
    assert L.dist_init_many(out, 1, gens, n, K, f, None) == -1
    assert L.dist_init_many(None, 0, None, None, None, None, None) == 0
    assert dist.dist_init_many([]) == ([], [])


def test_iso_walk_setting_without_device():
    saved = dist.dist_get_iso_walk()
    try:
        for mode in (1, 2, 0):
            dist.dist_set_iso_walk(mode)
            assert dist.dist_get_iso_walk() == mode
        with pytest.raises(dist.DistError) as e:
            dist.dist_set_iso_walk(3)
        assert e.value.code == -1
        with pytest.raises(dist.DistError):
            dist.dist_set_iso_walk(-1)
    finally:
        dist.dist_set_iso_walk(saved)
