"""The C-ABI library builds, loads without a GPU and exports every function
declared in include/chl.h; argument errors are reported before any GPU work."""
import ctypes as C
import os
import re

import pytest

import paper_1907_00140_gb300 as chl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "chl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(chl_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    chl.build()
    return chl.lib()


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert {"chl_build", "chl_query", "chl_labels_free", "chl_last_error"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name


def test_version(lib):
    assert "sm_103a" in chl.chl_version()


def test_null_arguments_are_einval(lib):
    assert lib.chl_build(None, None, None, None, None) == chl.CHL_EINVAL
    out = C.c_void_p()
    assert lib.chl_build(None, None, None, None, C.byref(out)) == chl.CHL_EINVAL
    assert "NULL" in chl.chl_last_error()
    g = chl.chl_csr(0, 0, None, None, None, 0)
    assert lib.chl_build(C.byref(g), C.c_void_p(1), None, None, C.byref(out)) == chl.CHL_EINVAL
    assert out.value is None
    assert lib.chl_query(None, None, 0, None, 0, None) == chl.CHL_EINVAL
    assert lib.chl_labels_info(None, None, None, None) == chl.CHL_EINVAL
    assert lib.chl_tune(None, None, None, None, None, None) == chl.CHL_EINVAL
    lib.chl_labels_free(None)
    assert lib.chl_labels_parents(None, None, 0, None) == chl.CHL_EINVAL
    assert lib.chl_path(None, None, 0, 0, None, None, 0, None) == chl.CHL_EINVAL
    # serving entry points
    assert lib.chl_server_create(None, None) == chl.CHL_EINVAL
    t = C.c_uint64()
    assert lib.chl_server_add_set(None, None, None) == chl.CHL_EINVAL
    assert lib.chl_server_submit_query(None, 0, None, 0, None, C.byref(t)) == chl.CHL_EINVAL
    assert lib.chl_server_submit_build(None, None, None, None, C.byref(t)) == chl.CHL_EINVAL
    assert lib.chl_server_wait(None, 1, 0.0, None, None) == chl.CHL_EINVAL
    assert lib.chl_server_replay(None, 0, None, None, None, None, None, None, None) == chl.CHL_EINVAL
    assert lib.chl_server_stats_get(None, None) == chl.CHL_EINVAL
    lib.chl_server_destroy(None)


def test_bad_server_options_are_einval(lib):
    h = C.c_void_p()
    for field, val in [("query_slots", -1), ("query_slots", 17), ("batching", 2),
                       ("build_workers", 99), ("max_batch", 1 << 27)]:
        o = chl.chl_server_opts()
        setattr(o, field, val)
        assert lib.chl_server_create(C.byref(o), C.byref(h)) == chl.CHL_EINVAL, field
        assert h.value is None


def test_bad_options_are_einval(lib):
    g = chl.chl_csr(4, 0, 1, None, None, chl.CHL_MEM_HOST)
    out = C.c_void_p()
    for field, val in [("common_hubs", 65), ("threads_per_tree", 48), ("threads_per_tree", 96), ("threads_per_tree", 2048), ("window_buckets", 1), ("mode", 3),
                       ("root_end", 9), ("slots", -1), ("flags", 16), ("pruned_bucket_delta", -2),
                       ("psi_threshold", -1.0), ("psi_threshold", float("nan")),
                       ("pruned_threads_per_tree", 48), ("pruned_threads_per_tree", 2048)]:
        o = chl.chl_build_opts()
        setattr(o, field, val)
        assert lib.chl_build(C.byref(g), C.c_void_p(1), C.byref(o), None, C.byref(out)) == chl.CHL_EINVAL, field


def test_no_fallback_without_library(tmp_path, monkeypatch):
    monkeypatch.setattr(chl, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(chl, "_lib", None)
    with pytest.raises(RuntimeError):
        chl.lib()


def test_build_options_are_marshalled_by_field_type(monkeypatch):
    """build_labels passes float options as floats and integer options as
    integers, and rejects unknown names (no GPU: chl_build is intercepted)."""
    import numpy as np
    seen = {}

    def fake_build(csr, rank_ptr, opts, stream):
        seen["opts"] = opts
        raise RuntimeError("intercepted")

    monkeypatch.setattr(chl, "chl_build", fake_build)

    class G:
        n = 2
        row_ptr = np.array([0, 1, 2], np.uint64)
        col = np.array([1, 0], np.uint32)
        w = np.array([3, 3], np.uint32)

    rank = np.array([1, 0], np.uint32)
    with pytest.raises(RuntimeError, match="intercepted"):
        chl.build_labels(G, rank, psi_threshold=0.5, bucket_delta=7, slots=3)
    o = seen["opts"]
    assert abs(o.psi_threshold - 0.5) < 1e-7 and o.bucket_delta == 7 and o.slots == 3
    with pytest.raises(TypeError):
        chl.build_labels(G, rank, no_such_option=1)


class LabelsMirror(C.Structure):
    """The library's handle layout (struct chl_labels in csrc/chl_common.cuh),
    for forging handles in tests only."""
    _fields_ = [("n", C.c_uint32), ("total", C.c_uint64), ("offsets", C.c_void_p),
                ("hub", C.c_void_p), ("hubpos", C.c_void_p), ("dist", C.c_void_p),
                ("parent", C.c_void_p), ("bytes", C.c_uint64), ("stats", chl.chl_build_stats),
                ("device", C.c_int)]


def test_forged_handle_is_refused_before_use(lib):
    """Every call that takes labels checks the handle's device first: a handle
    whose arrays are all null and whose device is not the current one comes
    back with an error (CHL_ECUDA without a GPU, CHL_EINVAL with one) instead
    of a dereference."""
    import numpy as np
    forged = LabelsMirror(n=4, total=0, parent=1, device=12345)
    h = C.addressof(forged)
    pairs = np.array([[0, 1]], np.uint32)
    out = np.zeros(1, np.uint32)
    offs = np.zeros(5, np.uint64)
    lens = np.zeros(1, np.uint32)
    for st in (lib.chl_query(h, pairs.ctypes.data, 1, out.ctypes.data, chl.CHL_MEM_HOST, None),
               lib.chl_query_noalloc(h, pairs.ctypes.data, 1, out.ctypes.data, chl.CHL_MEM_HOST, None),
               lib.chl_path(h, pairs.ctypes.data, 1, 0, None, lens.ctypes.data, chl.CHL_MEM_HOST, None),
               lib.chl_labels_copy(h, offs.ctypes.data, None, None, chl.CHL_MEM_HOST, None),
               lib.chl_labels_parents(h, out.ctypes.data, chl.CHL_MEM_HOST, None)):
        assert st in (chl.CHL_EINVAL, chl.CHL_ECUDA)
