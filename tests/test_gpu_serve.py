"""Serving loop (chl_server_*): every answer and every build is the same when
served alone and when served in a mix of label sets, concurrent builds,
batching modes and open-loop replays; answers equal the oracle's."""
import time

import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1907_00140_gb300 as chl  # noqa: E402
from test_gpu_parity import DG, dev  # noqa: E402


@pytest.fixture(scope="module")
def sets():
    """Two resident label sets (scale-free and grid) with oracle labels."""
    chl.build()
    out = []
    for g, rank in (W.load("ba2k"), (lambda g: (g, W.spt_count_rank(g, 32, seed=64)))(W.grid(64, 806, seed=64))):
        L = chl.build_labels(DG(g), dev(rank))
        ref = O.build_labels(g, rank, "plant", threads=8)
        out.append((g, rank, L, ref))
    return out


def alone(L, pairs):
    return L.query(np.ascontiguousarray(pairs, np.uint32))


def test_queries_same_alone_and_in_mix(sets):
    rng = np.random.default_rng(5)
    S = chl.Server(query_slots=3, max_batch=1 << 16)
    ids = [S.add_set(L) for _, _, L, _ in sets]
    reqs = []
    for i in range(300):
        k = int(rng.integers(0, 2))
        g = sets[k][0]
        q = int(rng.integers(1, 400))
        pairs = rng.integers(0, g.n, size=(q, 2)).astype(np.uint32)
        reqs.append((k, pairs, S.submit_query(ids[k], pairs)))
    # builds submitted into the same mix
    bg = [W.barabasi_albert(3000 + 1000 * j, 3 + j, seed=200 + j, wlo=1, whi=100) for j in range(2)]
    br = [W.degree_rank(g) for g in bg]
    bt = [S.submit_build(g, r) for g, r in zip(bg, br)]
    for _ in range(200):  # more queries while the builds run
        k = int(rng.integers(0, 2))
        pairs = rng.integers(0, sets[k][0].n, size=(64, 2)).astype(np.uint32)
        reqs.append((k, pairs, S.submit_query(ids[k], pairs)))
    for k, pairs, t in reqs:
        got, lat = S.wait(t)
        assert lat >= 0
        g, rank, L, ref = sets[k]
        assert np.array_equal(got, alone(L, pairs))
        assert np.array_equal(got, O.query(ref, rank, pairs))
    for g, r, t in zip(bg, br, bt):
        Lm, _ = S.wait(t)
        La = chl.build_labels(g, r)
        for x, y in zip(Lm.to_numpy(), La.to_numpy()):
            assert np.array_equal(x, y)
        ref = O.build_labels(g, r, "plant", threads=8)
        off, hub, dist = Lm.to_numpy()
        assert np.array_equal(off, ref.offsets) and np.array_equal(hub, ref.hub)
        assert np.array_equal(dist, ref.dist)
    st = S.stats()
    assert st["builds_done"] == 2 and st["batches"] >= 1 and st["pairs"] > 0
    S.close()


@pytest.mark.parametrize("batching", [0, 1])
def test_replay_open_loop(sets, batching):
    rng = np.random.default_rng(11 + batching)
    nreq = 2000
    rate = 2e5  # requests per second
    arr = np.cumsum(rng.exponential(1.0 / rate, nreq))
    set_of = rng.integers(0, 2, nreq).astype(np.uint32)
    sizes = rng.integers(1, 16, nreq)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    pairs = np.empty((int(off[-1]), 2), np.uint32)
    for i in range(nreq):
        n = sets[set_of[i]][0].n
        pairs[off[i]:off[i + 1]] = rng.integers(0, n, size=(sizes[i], 2))
    S = chl.Server(batching=batching)
    for _, _, L, _ in sets:
        S.add_set(L)
    out, lat, wall = S.replay(arr, set_of, off, pairs)
    assert (lat >= 0).all() and wall >= arr[-1] * 0.99
    for k in (0, 1):
        sel = np.repeat(set_of == k, sizes)
        g, rank, L, ref = sets[k]
        assert np.array_equal(out[sel], alone(L, pairs[sel]))
    st = S.stats()
    if batching == 1:
        assert st["batches"] == nreq           # plain: one launch per request
    assert st["pairs"] == int(off[-1])
    S.close()


def test_build_admission_by_memory_budget():
    """With a budget below two builds' estimates, builds run one at a time and
    still produce the labels they produce alone."""
    gs = [W.barabasi_albert(4000, 3, seed=300 + j, wlo=1, whi=100) for j in range(3)]
    rs = [W.degree_rank(g) for g in gs]
    S = chl.Server(build_workers=3, build_budget=1)  # only one admitted at a time
    ts = [S.submit_build(g, r) for g, r in zip(gs, rs)]
    for g, r, t in zip(gs, rs, ts):
        Lm, _ = S.wait(t)
        ref = O.build_labels(g, r, "plant", threads=8)
        off, hub, dist = Lm.to_numpy()
        assert np.array_equal(off, ref.offsets) and np.array_equal(hub, ref.hub)
        assert np.array_equal(dist, ref.dist)
    st = S.stats()
    assert st["builds_done"] == 3
    S.close()


def test_rejects_bad_requests(sets):
    S = chl.Server()
    k = S.add_set(sets[0][2])
    n = sets[0][0].n
    with pytest.raises(chl.ChlError) as e:
        S.submit_query(k, np.array([[0, n]], np.uint32))
    assert e.value.status == chl.CHL_EINVAL
    with pytest.raises(chl.ChlError) as e:
        S.submit_query(k + 5, np.array([[0, 1]], np.uint32))
    assert e.value.status == chl.CHL_EINVAL
    with pytest.raises(chl.ChlError) as e:
        S.wait(12345)
    assert e.value.status == chl.CHL_EINVAL
    t = S.submit_query(k, np.array([[0, 1]], np.uint32))
    got, _ = S.wait(t)
    assert got.tolist() == alone(sets[0][2], np.array([[0, 1]], np.uint32)).tolist()
    S.close()
