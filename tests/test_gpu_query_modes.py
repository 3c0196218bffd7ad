"""Query modes of the paper's Sec. 6 on one GPU, against the oracle.

- Hub-partitioned labels (QFDL-style): labels built over disjoint root ranges
  are the canonical labels split by hub (trees are independent, Sec. 5.2); a
  query takes the minimum of the partial merges, and must equal the oracle's
  answer over the whole labeling.
- Grouped batches (QDOL-style): the batch is sorted by the vertex blocks its
  pairs read and the answers are put back in arrival order; the answers must
  be those of the plain merge, pair for pair.
Both also run inside the serving loop (a partitioned set; query_order = 1).
All distances are integers: comparisons are exact.
"""
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


def graphs():
    g, r = W.load("ba2k")
    yield "ba2k", g, r
    g = W.grid(64, 800, seed=64)
    yield "grid64", g, W.spt_count_rank(g, 32, seed=64)


CASES = list(graphs())


def pairs_for(g, q, seed):
    p = W.uniform_pairs(g.n, q, seed)
    p[:50, 1] = p[:50, 0]  # u == v
    p[50:100] = p[50:100, ::-1]  # both orders
    return np.ascontiguousarray(p)


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request):
    chl.build()
    name, g, rank = request.param
    ref = O.build_labels(g, rank, "plant")
    return name, g, rank, ref


def split_ranges(n):
    cuts = sorted({0, min(n, 16), min(n, 150), n // 3, n})
    return list(zip(cuts[:-1], cuts[1:]))


def test_partitioned_queries_equal_oracle(case):
    name, g, rank, ref = case
    parts = [chl.build_labels(DG(g), dev(rank), root_begin=b, root_end=e) for b, e in split_ranges(g.n)]
    pos = g.n - 1 - rank.astype(np.int64)
    for (b, e), L in zip(split_ranges(g.n), parts):
        off, hub, dist = L.to_numpy()
        keep = (pos[ref.hub] >= b) & (pos[ref.hub] < e)
        assert np.array_equal(hub, ref.hub[keep]) and np.array_equal(dist, ref.dist[keep])
    pairs = pairs_for(g, 30000, seed=21)
    want = O.query(ref, rank, pairs)
    got_d = chl.query_partitioned(parts, dev(pairs)).cpu().numpy().view(np.uint32)
    got_h = chl.query_partitioned(parts, pairs)
    assert np.array_equal(got_d, want) and np.array_equal(got_h, want)
    bad = pairs.copy()
    bad[7, 0] = g.n
    with pytest.raises(chl.ChlError) as e:
        chl.query_partitioned(parts, bad)
    assert e.value.status == chl.CHL_EINVAL
    for L in parts:
        L.free()


def test_grouped_queries_equal_oracle(case):
    name, g, rank, ref = case
    L = chl.build_labels(DG(g), dev(rank))
    for q, seed in ((1, 3), (777, 4), (50000, 5)):
        pairs = pairs_for(g, q, seed) if q > 100 else W.uniform_pairs(g.n, q, seed)
        want = O.query(ref, rank, pairs)
        got_d = L.query(dev(pairs), grouped=True).cpu().numpy().view(np.uint32)
        got_h = L.query(pairs, grouped=True)
        assert np.array_equal(got_d, want) and np.array_equal(got_h, want)
    L.free()


@pytest.mark.parametrize("order", [0, 1])
def test_server_partitioned_set_and_grouped_batches(case, order):
    name, g, rank, ref = case
    L = chl.build_labels(DG(g), dev(rank))
    parts = [chl.build_labels(DG(g), dev(rank), root_begin=b, root_end=e) for b, e in split_ranges(g.n)]
    S = chl.Server(query_order=order)
    s_whole = S.add_set(L)
    s_part = S.add_partitioned_set(parts)
    tickets = []
    for k, q in enumerate((10, 5000, 20000, 70000)):  # the larger batches are grouped
        pairs = pairs_for(g, q, 40 + k) if q > 100 else W.uniform_pairs(g.n, q, 40 + k)
        want = O.query(ref, rank, pairs)
        tickets.append((S.submit_query(s_whole, pairs), want))
        tickets.append((S.submit_query(s_part, pairs), want))
    for t, want in tickets:
        got, _lat = S.wait(t, timeout=60.0)
        assert np.array_equal(got, want)
    # a replay mixing both sets
    rng = np.random.default_rng(3)
    nreq = 400
    sizes = rng.integers(1, 300, nreq)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    pairs = W.uniform_pairs(g.n, int(off[-1]), seed=77)
    set_of = rng.integers(0, 2, nreq).astype(np.uint32)
    arr = np.cumsum(rng.exponential(2e-5, nreq))
    ans, lat, wall = S.replay(arr, np.where(set_of == 0, s_whole, s_part), off, pairs)
    assert np.array_equal(ans, O.query(ref, rank, pairs))
    S.close()
    for x in parts:
        x.free()
    L.free()
