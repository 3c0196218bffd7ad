"""Failure paths of the C ABI on the GPU, made without faulting the GPU.

- A tree that needs more expansion rounds than round_limit stops the build
  with CHL_ETIMEOUT (the kernel sets a flag and returns; nothing waits), and
  the CUDA context stays usable: the next build is bit-exact.
- A label buffer larger than device memory fails its allocation: CHL_ENOMEM.
- A labels handle whose recorded device is not the current one is refused
  with CHL_EINVAL before any of its arrays is touched (a forged handle with
  null arrays; the mirror of the handle's layout is checked against a real one).
- A query batch whose launch fails (a host-side fake of the failing launch,
  CHL_FAULT_QUERY_BATCH) finishes its requests with CHL_ECUDA; the server frees
  the slot and keeps serving.
"""
import ctypes as C
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1907_00140_gb300 as chl  # noqa: E402

from test_gpu_parity import DG, dev, gpu_labels, assert_same  # noqa: E402
from test_abi_cpu import LabelsMirror  # noqa: E402


@pytest.fixture(scope="module")
def ba():
    chl.build()
    g, rank = W.load("ba2k")
    return g, rank, O.build_labels(g, rank, "plant")


def test_round_limit_is_etimeout_and_context_survives(ba):
    g, rank, ref = ba
    with pytest.raises(chl.ChlError) as e:
        chl.build_labels(DG(g), dev(rank), round_limit=2)
    assert e.value.status == chl.CHL_ETIMEOUT
    torch.cuda.synchronize()
    L, off, hub, dist = gpu_labels(g, rank)
    assert_same(ref, off, hub, dist)
    L.free()


def test_unsatisfiable_label_buffer_is_enomem(ba):
    g, rank, ref = ba
    with pytest.raises(chl.ChlError) as e:
        chl.build_labels(DG(g), dev(rank), label_capacity=1 << 42)
    assert e.value.status == chl.CHL_ENOMEM
    L, off, hub, dist = gpu_labels(g, rank)
    assert_same(ref, off, hub, dist)
    L.free()


def test_handle_of_another_device_is_refused(ba):
    g, rank, ref = ba
    L, off, hub, dist = gpu_labels(g, rank)
    real = LabelsMirror.from_buffer_copy(C.string_at(L.handle, C.sizeof(LabelsMirror)))
    n, total, _ = chl.chl_labels_info(L.handle)
    assert (real.n, real.total, real.device) == (n, total, torch.cuda.current_device())
    forged = LabelsMirror(n=4, total=0, parent=1, device=torch.cuda.current_device() + 1)
    h = C.addressof(forged)
    lib = chl.lib()
    pairs = np.array([[0, 1]], np.uint32)
    out = np.zeros(1, np.uint32)
    lens = np.zeros(1, np.uint32)
    offs = np.zeros(5, np.uint64)
    k = C.c_uint32()
    S = chl.Server()
    for name, call in [
        ("chl_query", lambda: lib.chl_query(h, pairs.ctypes.data, 1, out.ctypes.data, chl.CHL_MEM_HOST, None)),
        ("chl_query_noalloc", lambda: lib.chl_query_noalloc(h, pairs.ctypes.data, 1, out.ctypes.data,
                                                            chl.CHL_MEM_HOST, None)),
        ("chl_path", lambda: lib.chl_path(h, pairs.ctypes.data, 1, 0, None, lens.ctypes.data,
                                          chl.CHL_MEM_HOST, None)),
        ("chl_labels_copy", lambda: lib.chl_labels_copy(h, offs.ctypes.data, None, None, chl.CHL_MEM_HOST, None)),
        ("chl_server_add_set", lambda: lib.chl_server_add_set(S.handle, h, C.byref(k))),
    ]:
        assert call() == chl.CHL_EINVAL, name
        assert b"device" in lib.chl_last_error(), name
    S.close()
    # the real handle still answers
    assert np.array_equal(L.query(dev(pairs)).cpu().numpy().view(np.uint32), O.query(ref, rank, pairs))
    L.free()


def test_failed_query_batch_is_ecuda_and_server_recovers(ba, monkeypatch):
    g, rank, ref = ba
    L, *_ = gpu_labels(g, rank)
    monkeypatch.setenv("CHL_FAULT_QUERY_BATCH", "1")
    S = chl.Server()
    monkeypatch.delenv("CHL_FAULT_QUERY_BATCH")
    sid = S.add_set(L)
    pairs = W.uniform_pairs(g.n, 500, seed=9)
    t = S.submit_query(sid, pairs)
    with pytest.raises(chl.ChlError) as e:
        S.wait(t, timeout=30.0)
    assert e.value.status == chl.CHL_ECUDA
    want = O.query(ref, rank, pairs)
    for _ in range(3):
        got, _lat = S.wait(S.submit_query(sid, pairs), timeout=30.0)
        assert np.array_equal(got, want)
    S.close()
    L.free()
