"""The C-ABI library builds, loads and exports every symbol include/tl.h declares.

No compute call here: these run without a GPU.
"""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2203_04774_gb300 as tl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "tl.h")).read()
    return sorted(set(re.findall(r"TL_EXPORT\s+[\w\s\*]+?\b(tl_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()
    return tl.lib()


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for must in ("tl_graph_load", "tl_order_apply", "tl_list_triangles", "tl_cost",
                 "tl_graph_free", "tl_last_error", "tl_count_hash"):
        assert must in names


def test_library_exports_every_declared_symbol(built):
    exported = subprocess.run(["nm", "-D", "--defined-only", tl.LIB_PATH], capture_output=True,
                              text=True, check=True).stdout
    syms = {line.split()[-1] for line in exported.splitlines() if " T " in line}
    for name in _declared_symbols():
        assert name in syms, name
        assert hasattr(built, name)
    # the binding wraps exactly the declared names
    assert set(tl.SIGNATURES) == set(_declared_symbols())


def test_version_and_error_strings_without_gpu(built):
    assert built.tl_version().decode().startswith("tl ")
    assert built.tl_last_error() is not None


def test_null_arguments_rejected_without_gpu(built):
    # argument checks come before any device work
    assert built.tl_graph_load(None, 10, None, 0, 0, None) == tl.TL_EINVAL
    h = ctypes.c_void_p()
    assert built.tl_graph_load(ctypes.byref(h), 0, None, 0, 0, None) == tl.TL_EINVAL
    assert built.tl_cost(None, 0, None) == tl.TL_EINVAL
    assert built.tl_list_triangles(None, 0, 1 << 30, None, None, None) == tl.TL_EINVAL
    built.tl_graph_free(None)


def test_no_device_is_an_error_not_a_fallback(built):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np
    e = np.array([[0, 1], [1, 2], [0, 2]], dtype=np.uint32)
    h = ctypes.c_void_p()
    st = built.tl_graph_load(ctypes.byref(h), 3, e.ctypes.data, 3, 0, None)
    assert st == tl.TL_ECUDA


def test_union_and_server_arguments_rejected_without_gpu(built):
    h = ctypes.c_void_p()
    n = (ctypes.c_uint32 * 2)(3, 0)
    m = (ctypes.c_uint64 * 2)(0, 0)
    assert built.tl_graph_load_parts(ctypes.byref(h), 0, n, m, None, 0, None) == tl.TL_EINVAL
    assert built.tl_graph_load_parts(ctypes.byref(h), 2, n, m, None, 0, None) == tl.TL_EINVAL
    assert built.tl_graph_union(ctypes.byref(h), None, None, 1, None) == tl.TL_EINVAL
    for cfg in (tl.ServerConfig(1 << 30, 0, 1, 64 << 20), tl.ServerConfig(1 << 30, 8, 0, 64 << 20),
                tl.ServerConfig(1 << 30, 8, 1, 1 << 20)):
        assert built.tl_server_create(ctypes.byref(h), ctypes.byref(cfg)) == tl.TL_EINVAL
    assert built.tl_server_create(ctypes.byref(h), None) == tl.TL_EINVAL
    built.tl_server_free(None)
    assert built.tl_count_hash_parts(None, 0, 0, None) != 0


def test_tuning_defaults_and_argument_checks_without_gpu(built):
    t = tl.tl_default_tuning()
    assert t == {"small_max_p": 32, "medium_max_p": 1024, "narrow_max_p": 256,
                 "mid_max_p": 2048, "warp_work": 4096, "narrow_piece": 1 << 14,
                 "mid_piece": 1 << 16,
                 "large_per_p": 64, "large_min": 1 << 16, "large_max": 1 << 22,
                 "narrow_keep_mib": 0, "narrow_cold_first": 0, "large_hash_max_p": 16384}
    assert built.tl_set_tuning(None, None) == tl.TL_EINVAL
    out = tl.Tuning()
    assert built.tl_get_tuning(None, ctypes.byref(out)) == tl.TL_EINVAL
