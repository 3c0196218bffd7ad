"""GPU parity: labels and query answers of libchl.so against the CPU oracle.

All arithmetic is integer and the canonical labeling is unique for a fixed
rank (Sec. 1; PLaNT, DGLL and Hybrid produce the same labels, Sec. 7.3), so
every comparison is bit-exact: offsets, hub ids, distances and query answers.
Calls go through the C ABI (ctypes binding) with device tensors, except where
the host-memory path itself is under test.
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

from test_oracle import from_edges, tiny_cases, read_fixture  # noqa: E402

DEV = torch.device("cuda:0")
U32MAX = np.iinfo(np.uint32).max


@pytest.fixture(scope="module", autouse=True)
def _built():
    chl.build()
    chl.lib()


def dev(a):
    a = np.ascontiguousarray(a)
    v = a.view(np.int64) if a.dtype == np.uint64 else a.view(np.int32)
    return torch.from_numpy(v).to(DEV)


class DG:
    """Graph arrays as device tensors."""

    def __init__(self, g):
        self.n = g.n
        self.row_ptr = dev(g.row_ptr)
        self.col = dev(g.col)
        self.w = dev(g.w)


def gpu_labels(g, rank, host=False, **opts):
    L = chl.build_labels(g if host else DG(g), rank if host else dev(rank), **opts)
    off, hub, dist = L.to_numpy()
    return L, off, hub, dist


def assert_same(ref, off, hub, dist):
    assert np.array_equal(off, ref.offsets), "offsets"
    assert np.array_equal(hub, ref.hub), "hub"
    assert np.array_equal(dist, ref.dist), "dist"


# ------------------------------------------------------------------ tiny graphs
@pytest.mark.parametrize("name,g,rank", tiny_cases(), ids=[c[0] for c in tiny_cases()])
def test_tiny_bit_exact(name, g, rank):
    ref = O.build_labels(g, rank, "canonical")
    L, off, hub, dist = gpu_labels(g, rank)
    assert_same(ref, off, hub, dist)
    n = g.n
    u, v = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    pairs = np.stack([u.ravel(), v.ravel()], 1).astype(np.uint32)
    got = L.query(dev(pairs)).cpu().numpy().view(np.uint32)
    assert np.array_equal(got, O.query(ref, rank, pairs))


@pytest.mark.parametrize("fixture", ["a1_counterexample.txt", "fig1_tie_fragment.txt"])
def test_fixtures(fixture):
    g, rank, _, _ = read_fixture(fixture)
    ref = O.build_labels(g, rank, "canonical")
    _, off, hub, dist = gpu_labels(g, rank)
    assert_same(ref, off, hub, dist)


def test_single_vertex():
    g = from_edges(1, [])
    rank = np.zeros(1, np.uint32)
    L, off, hub, dist = gpu_labels(g, rank)
    assert off.tolist() == [0, 1] and hub.tolist() == [0] and dist.tolist() == [0]
    assert L.query(np.array([[0, 0]], np.uint32)).tolist() == [0]


def test_disconnected_and_special_queries():
    g = from_edges(6, [(0, 1, 4), (1, 2, 4), (3, 4, 7), (4, 5, 1)])
    rank = np.array([5, 4, 3, 2, 1, 0], np.uint32)
    L, *_ = gpu_labels(g, rank)
    q = np.array([[2, 2], [0, 2], [0, 3], [5, 3], [4, 4]], np.uint32)
    assert L.query(q).tolist() == [0, 8, U32MAX, 8, 0]
    assert L.query(np.zeros((0, 2), np.uint32)).tolist() == []


# ------------------------------------------------------------------ ba2k (config 1) in full
@pytest.fixture(scope="module")
def ba2k():
    g, rank = W.load("ba2k")
    return g, rank, O.build_labels(g, rank, "plant", threads=4)


def test_ba2k_labels_and_queries(ba2k):
    g, rank, ref = ba2k
    L, off, hub, dist = gpu_labels(g, rank)
    assert_same(ref, off, hub, dist)
    pairs = W.query_pairs(g, 100_000, seed=2)
    got = L.query(dev(pairs)).cpu().numpy().view(np.uint32)
    assert np.array_equal(got, O.query(ref, rank, pairs, threads=4))
    st = L.stats()
    assert st["trees"] == g.n and st["labels"] == ref.total


def test_ba2k_host_memory_path(ba2k):
    g, rank, ref = ba2k
    L, off, hub, dist = gpu_labels(g, rank, host=True)
    assert_same(ref, off, hub, dist)
    pairs = W.query_pairs(g, 5000, seed=4)
    assert np.array_equal(L.query(pairs), O.query(ref, rank, pairs))


@pytest.mark.parametrize("opts", [
    dict(threads_per_tree=32), dict(threads_per_tree=64), dict(threads_per_tree=256),
    dict(threads_per_tree=512), dict(threads_per_tree=1024), dict(bucket_delta=1),
    dict(bucket_delta=1000),
    dict(window_buckets=2), dict(window_buckets=64, bucket_delta=1), dict(slots=1),
    dict(slots=7, threads_per_tree=32), dict(label_capacity=1), dict(mode=1),
    dict(mode=1, threads_per_tree=64), dict(flags=chl.CHL_FLAG_WIDE_KEYS),
    dict(common_hubs=-1), dict(common_hubs=1), dict(common_hubs=4), dict(common_hubs=64),
    dict(common_hubs=64, bucket_delta=5, threads_per_tree=128),
    dict(mode=1, common_hubs=8), dict(common_hubs=3, flags=chl.CHL_FLAG_WIDE_KEYS),
    dict(flags=chl.CHL_FLAG_WIDE_KEYS, threads_per_tree=64, bucket_delta=3),
], ids=lambda o: ",".join(f"{k}={v}" for k, v in o.items()))
def test_ba2k_launch_configurations(ba2k, opts):
    g, rank, ref = ba2k
    _, off, hub, dist = gpu_labels(g, rank, **opts)
    assert_same(ref, off, hub, dist)


def test_heavy_weights_take_wide_keys():
    """w_max * n above 2^31 - 1: the build must switch to 8-byte keys and stay
    exact for distances above 2^31 (still below the 2^32 - 1 limit)."""
    rng = np.random.default_rng(77)
    g0 = W.barabasi_albert(300, 2, seed=77, wlo=1, whi=100)
    eu, ev, _ = g0.edges()
    edges = [(int(a), int(b), int(rng.integers(1 << 26, 1 << 27))) for a, b in zip(eu, ev)]
    g = from_edges(g0.n, edges)
    rank = W.degree_rank(g)
    ref = O.build_labels(g, rank, "canonical")
    assert not ref.overflow and int(ref.dist.max()) > (1 << 28)
    for opts in (dict(), dict(bucket_delta=1 << 24)):
        _, off, hub, dist = gpu_labels(g, rank, **opts)
        assert_same(ref, off, hub, dist)


def test_tuned_parameters_are_exact(ba2k):
    g, rank, ref = ba2k
    opts, rep = chl.tune(DG(g), dev(rank))
    assert rep["trials"] >= 3 and rep["sample_roots"] >= 1 and rep["best_tree_ms"] > 0
    assert opts["threads_per_tree"] in (128, 256, 512, 1024) and opts["bucket_delta"] >= 1
    _, off, hub, dist = gpu_labels(g, rank, **opts)
    assert_same(ref, off, hub, dist)
    fixed, _ = chl.tune(DG(g), dev(rank), bucket_delta=7)
    assert fixed["bucket_delta"] == 7


def test_common_label_table_prunes(ba2k):
    """The table (Sec. 5.3) cuts expansions and arcs but not one label."""
    g, rank, ref = ba2k
    G, R = DG(g), dev(rank)
    off_ = chl.build_labels(G, R, common_hubs=-1)
    on_ = chl.build_labels(G, R, common_hubs=16)
    a, b = off_.stats(), on_.stats()
    assert a["pruned"] == 0 and b["pruned"] > 0
    assert b["arcs"] < a["arcs"] and b["labels"] == a["labels"] == ref.total
    assert_same(ref, *on_.to_numpy())


def test_root_ranges_partition_labels_by_hub(ba2k):
    g, rank, ref = ba2k
    n = g.n
    order = np.empty(n, np.uint32)
    order[n - 1 - rank.astype(np.int64)] = np.arange(n, dtype=np.uint32)
    for rb, re in [(0, 1), (0, 64), (64, 700), (700, n), (n - 1, n), (5, 5), (10, 20), (16, 17)]:
        want = O.build_labels(g, rank, "plant", roots=order[rb:re])
        _, off, hub, dist = gpu_labels(g, rank, root_begin=rb, root_end=re)
        assert_same(want, off, hub, dist)


def test_repeated_single_slot_builds(ba2k):
    """One CTA runs every tree back to back on the same slot state, with
    narrow buckets (many rounds per bucket): the configuration most exposed to
    ordering races between rounds, buckets and consecutive trees."""
    g, rank, ref = ba2k
    G, R = DG(g), dev(rank)
    for _ in range(12):
        L = chl.build_labels(G, R, slots=1, bucket_delta=3)
        assert_same(ref, *L.to_numpy())
        L.free()


def test_deterministic(ba2k):
    g, rank, _ = ba2k
    a = gpu_labels(g, rank)[1:]
    b = gpu_labels(g, rank, slots=3)[1:]
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


# ------------------------------------------------------------------ mid-size families, several tiles
@pytest.mark.parametrize("family", ["rmat13", "grid64", "ba_w3"])
def test_mid_size_families(family):
    if family == "rmat13":
        g = W.rmat(13, 16, seed=13, whi=255)
        rank = W.degree_rank(g)
    elif family == "grid64":
        g = W.grid(64, 806, seed=64)
        rank = W.spt_count_rank(g, 32, seed=64)
    else:
        g = W.barabasi_albert(6000, 4, seed=5, wlo=1, whi=3)  # heavy ties
        rank = W.degree_rank(g)
    ref = O.build_labels(g, rank, "plant", threads=8)
    for opts in (dict(), dict(threads_per_tree=64, bucket_delta=3), dict(label_capacity=1000)):
        L, off, hub, dist = gpu_labels(g, rank, **opts)
        assert_same(ref, off, hub, dist)
    pairs = W.query_pairs(g, 50_000, seed=9)
    assert np.array_equal(L.query(dev(pairs)).cpu().numpy().view(np.uint32),
                          O.query(ref, rank, pairs, threads=8))


# ------------------------------------------------------------------ input validation
def _status(g, rank):
    with pytest.raises(chl.ChlError) as e:
        chl.build_labels(g, rank)
    return e.value.status


def test_rejects_malformed_inputs():
    g = from_edges(4, [(0, 1, 2), (1, 2, 3), (2, 3, 4)])
    rank = np.array([0, 1, 2, 3], np.uint32)
    assert _status(g, np.array([0, 1, 1, 3], np.uint32)) == chl.CHL_EINVAL   # not a permutation
    assert _status(g, np.array([0, 1, 2, 4], np.uint32)) == chl.CHL_EINVAL   # out of range
    bad = from_edges(4, [(0, 1, 2), (1, 2, 3), (2, 3, 4)])
    bad.w = bad.w.copy(); bad.w[0] = 0
    assert _status(bad, rank) == chl.CHL_EINVAL                               # zero weight
    asym = from_edges(4, [(0, 1, 2), (1, 2, 3), (2, 3, 4)])
    asym.w = asym.w.copy(); asym.w[1] = 9                                     # arc 1->0 != 0->1
    assert _status(asym, rank) == chl.CHL_EINVAL
    unsorted = from_edges(4, [(0, 1, 2), (0, 2, 3), (2, 3, 4)])
    unsorted.col = unsorted.col.copy(); unsorted.col[[0, 1]] = unsorted.col[[1, 0]]
    assert _status(unsorted, rank) == chl.CHL_EINVAL
    row = from_edges(4, [(0, 1, 2), (1, 2, 3), (2, 3, 4)])
    row.row_ptr = row.row_ptr.copy(); row.row_ptr[2] = 99
    assert _status(row, rank) == chl.CHL_EINVAL


def test_asymmetric_arcs_found_in_a_large_graph(ba2k):
    """The symmetry check streams a fingerprint of the arcs and their
    reverses; an arc whose reverse differs in weight, or is missing, still
    comes back as CHL_EINVAL naming a vertex with such an arc."""
    g, rank, _ = ba2k
    W_ = type(g)
    heavy = W_(g.n, g.row_ptr, g.col, g.w.copy())
    heavy.w[len(g.w) // 2] += 1
    with pytest.raises(chl.ChlError) as e:
        chl.build_labels(heavy, rank)
    assert e.value.status == chl.CHL_EINVAL and "reverse arc" in str(e.value)
    # drop the last arc of a middle row: the row stays sorted, its reverse is left alone
    v = g.n // 2
    a, b = int(g.row_ptr[v]), int(g.row_ptr[v + 1])
    keep = np.ones(len(g.col), bool)
    keep[b - 1] = False
    row = g.row_ptr.copy()
    row[v + 1:] -= 1
    missing = W_(g.n, row, g.col[keep].copy(), g.w[keep].copy())
    with pytest.raises(chl.ChlError) as e:
        chl.build_labels(missing, rank)
    assert e.value.status == chl.CHL_EINVAL and "reverse arc" in str(e.value)
    # the unchanged graph passes the same check
    chl.build_labels(g, rank).free()


def test_distance_overflow_is_reported():
    big = 2 ** 31
    g = from_edges(4, [(0, 1, big), (1, 2, big), (2, 3, 5)])
    assert _status(g, np.array([3, 2, 1, 0], np.uint32)) == chl.CHL_EOVERFLOW


def test_query_rejects_bad_vertex(ba2k):
    g, rank, _ = ba2k
    L, *_ = gpu_labels(g, rank, root_end=10)
    with pytest.raises(chl.ChlError) as e:
        L.query(np.array([[0, g.n]], np.uint32))
    assert e.value.status == chl.CHL_EINVAL


def test_hybrid_phases_are_exact():
    """A scale-free build deep enough to pass the Psi switch prunes its later
    phases with the label table of the earlier ones (Sec. 5.2) and still equals
    the oracle; the single-phase build gives the same labels with more work."""
    g = W.rmat(14, 16, seed=14, wlo=1, whi=255)
    rank = W.degree_rank(g)
    ref = O.build_labels(g, rank, "plant", threads=16)
    G, R = DG(g), dev(rank)
    for opts in (dict(), dict(threads_per_tree=256), dict(threads_per_tree=1024, bucket_delta=2),
                 dict(flags=chl.CHL_FLAG_DENSE_ROOT_LABELS), dict(pruned_bucket_delta=1),
                 dict(pruned_bucket_delta=4096, flags=chl.CHL_FLAG_PARENTS), dict(psi_threshold=0.5),
                 dict(psi_threshold=8.0, label_capacity=1000), dict(pruned_threads_per_tree=256),
                 dict(threads_per_tree=512, pruned_threads_per_tree=64, slots=5)):
        L = chl.build_labels(G, R, **opts)
        st = L.stats()
        assert st["phases"] > 1, st
        # Psi alone (a threshold given) may switch later or not at all
        assert st["label_table_phases"] >= 1 or opts.get("psi_threshold", 0) > 1, st
        assert_same(ref, *L.to_numpy())
    one = chl.build_labels(G, R, flags=chl.CHL_FLAG_NO_HYBRID)
    s1 = one.stats()
    assert s1["phases"] == 1 and s1["label_table_phases"] == 0
    assert s1["arcs"] > st["arcs"]
    assert_same(ref, *one.to_numpy())
    # a root range that does not start at the top runs as one phase
    part = chl.build_labels(G, R, root_begin=10, root_end=3000)
    assert part.stats()["phases"] == 1
