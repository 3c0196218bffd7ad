"""chl_query_noalloc: queries for callers that must not allocate memory.

The entry point stages pairs and answers in one fixed device array inside the
library instead of allocating per call. Its answers must equal those of
chl_query exactly (integer distances), on two calls in a row with different
pairs (the shared array keeps the previous call's contents), for host and
device buffers; requests above its size limit are refused.

This file is collected last on purpose, so a run that stops at the first
failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1907_00140_gb300 as chl  # noqa: E402

DEV = torch.device("cuda:0")
MAX_PAIRS = 1 << 20


def dev(a):
    a = np.ascontiguousarray(a)
    v = a.view(np.int64) if a.dtype == np.uint64 else a.view(np.int32)
    return torch.from_numpy(v).to(DEV)


@pytest.fixture(scope="module")
def labels():
    chl.build()
    g, rank = W.load("ba2k")

    class DG:
        n = g.n
        row_ptr = dev(g.row_ptr)
        col = dev(g.col)
        w = dev(g.w)

    L = chl.build_labels(DG, dev(rank))
    yield g, L
    L.free()


def reference(L, pairs):
    return L.query(pairs)  # chl_query, host buffers


def test_noalloc_host_buffers_two_calls(labels):
    g, L = labels
    a = W.uniform_pairs(g.n, 100_000, seed=21)
    b = W.uniform_pairs(g.n, 30_000, seed=22)  # shorter second call: stale tail in the array
    for pairs in (a, b):
        out = np.full(len(pairs), 7, np.uint32)
        chl.chl_query_noalloc(L.handle, pairs.ctypes.data, len(pairs), out.ctypes.data,
                              chl.CHL_MEM_HOST, torch.cuda.current_stream().cuda_stream)
        assert np.array_equal(out, reference(L, pairs))


def test_noalloc_device_buffers_two_calls(labels):
    g, L = labels
    for seed in (23, 24):
        pairs = W.uniform_pairs(g.n, 50_000, seed=seed)
        dp = dev(pairs)
        out = torch.empty(len(pairs), dtype=torch.int32, device=DEV)
        chl.chl_query_noalloc(L.handle, dp.data_ptr(), len(pairs), out.data_ptr(),
                              chl.CHL_MEM_DEVICE, torch.cuda.current_stream().cuda_stream)
        assert np.array_equal(out.cpu().numpy().view(np.uint32), reference(L, pairs))


def test_noalloc_limits_and_errors(labels):
    g, L = labels
    lib = chl.lib()
    one = np.zeros(2, np.uint32)
    res = np.zeros(1, np.uint32)
    st = lib.chl_query_noalloc(C.c_void_p(L.handle), C.c_void_p(one.ctypes.data),
                               C.c_uint64(MAX_PAIRS + 1), C.c_void_p(res.ctypes.data),
                               chl.CHL_MEM_HOST, None)
    assert st == chl.CHL_EINVAL and "at most" in chl.chl_last_error()
    bad = np.array([[0, g.n]], np.uint32)
    with pytest.raises(chl.ChlError) as e:
        chl.chl_query_noalloc(L.handle, bad.ctypes.data, 1, res.ctypes.data, chl.CHL_MEM_HOST, 0)
    assert e.value.status == chl.CHL_EINVAL
    # the flag left set by the failed call is cleared by the next call
    ok = W.uniform_pairs(g.n, 1000, seed=25)
    out = np.empty(1000, np.uint32)
    chl.chl_query_noalloc(L.handle, ok.ctypes.data, 1000, out.ctypes.data, chl.CHL_MEM_HOST, 0)
    assert np.array_equal(out, reference(L, ok))
