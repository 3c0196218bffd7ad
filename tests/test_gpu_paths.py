"""Shortest-path recovery (CHL_FLAG_PARENTS, chl_path): the SPT parent stored
with every label and the paths followed from them are bit-identical to the
oracle's (highest-ranked shortest-path predecessor; canonical hub per pair),
and the labels themselves are unchanged by carrying parents."""
import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1907_00140_gb300 as chl  # noqa: E402
from test_gpu_parity import DG, dev, assert_same  # noqa: E402
from test_oracle import tiny_cases  # noqa: E402

PAR = chl.CHL_FLAG_PARENTS


def check(g, rank, pairs, max_len=64, **opts):
    ref = O.build_labels(g, rank, "plant", threads=8)
    L = chl.build_labels(DG(g), dev(rank), flags=PAR, **opts)
    assert_same(ref, *L.to_numpy())
    want_par = O.parents(g, rank, ref)
    assert np.array_equal(L.parents(), want_par)
    got, lens = L.paths(pairs, max_len=max_len)
    want = O.paths(ref, rank, want_par, pairs)
    for i, w in enumerate(want):
        assert int(lens[i]) == len(w), (i, pairs[i])
        k = min(len(w), max_len)
        assert got[i, :k].tolist() == w[:k], (i, pairs[i])
    return L


@pytest.mark.parametrize("name,g,rank", tiny_cases(), ids=[c[0] for c in tiny_cases()])
def test_tiny_parents_and_all_paths(name, g, rank):
    n = g.n
    pairs = np.array([(u, v) for u in range(n) for v in range(n)], np.uint32)
    check(g, rank, pairs)


@pytest.mark.parametrize("opts", [dict(), dict(common_hubs=-1), dict(bucket_delta=7, threads_per_tree=128),
                                  dict(mode=1), dict(slots=1)],
                         ids=lambda o: ",".join(f"{k}={v}" for k, v in o.items()) or "default")
def test_ba2k_parents_and_paths(opts):
    g, rank = W.load("ba2k")
    pairs = W.uniform_pairs(g.n, 5000, seed=8)
    check(g, rank, pairs, **opts)


@pytest.mark.parametrize("family", ["rmat12", "grid48"])
def test_mid_size_paths(family):
    if family == "rmat12":
        g = W.rmat(12, 8, seed=12, wlo=1, whi=50)
        rank = W.degree_rank(g)
    else:
        g = W.grid(48, 400, seed=48)
        rank = W.spt_count_rank(g, 16, seed=48)
    pairs = np.concatenate([W.uniform_pairs(g.n, 3000, seed=3), W.degree_pairs(g, 1000, seed=4)])
    check(g, rank, pairs, max_len=512)


def test_truncated_paths_and_errors():
    g, rank = W.load("ba2k")
    pairs = W.uniform_pairs(g.n, 200, seed=5)
    L = check(g, rank, pairs, max_len=2)  # lens keep the full length, 2 vertices written
    with pytest.raises(chl.ChlError) as e:
        L.paths(np.array([[0, g.n]], np.uint32))
    assert e.value.status == chl.CHL_EINVAL
    plain = chl.build_labels(DG(g), dev(rank))
    with pytest.raises(chl.ChlError) as e:
        plain.paths(pairs)
    assert e.value.status == chl.CHL_EINVAL
    # parents leave the distances unchanged
    for x, y in zip(plain.to_numpy(), L.to_numpy()):
        assert np.array_equal(x, y)
