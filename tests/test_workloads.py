"""Seeded input generators: structure, determinism and the stated recipes."""
import numpy as np
import pytest
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import connected_components

import workloads as W


def check_graph(g, wlo, whi):
    n = g.n
    row, col, w = g.row_ptr, g.col, g.w
    assert row[0] == 0 and (np.diff(row.astype(np.int64)) >= 0).all()
    src = np.repeat(np.arange(n), np.diff(row.astype(np.int64)))
    assert (col < n).all() and (src != col).all()                      # no self-loops
    for v in range(0, n, max(1, n // 500)):                             # sorted rows, no dupes
        r = col[row[v]:row[v + 1]]
        assert (np.diff(r.astype(np.int64)) > 0).all()
    A = csr_matrix((w.astype(np.float64), col.astype(np.int64), row.astype(np.int64)), shape=(n, n))
    assert (A != A.T).nnz == 0                                          # symmetric, equal weights
    assert connected_components(A, directed=False)[0] == 1
    assert w.min() >= wlo and w.max() <= whi


def test_ba2k_recipe():
    g, rank = W.load("ba2k")
    assert g.n == 2000 and g.m == 6 + 3 * 1996
    check_graph(g, 1, 100)
    assert sorted(rank.tolist()) == list(range(g.n))


def test_degree_rank_order():
    g, rank = W.load("ba2k")
    deg = g.degree()
    order = np.argsort(-rank.astype(np.int64))  # most important first
    for a, b in zip(order[:-1], order[1:]):
        assert deg[a] > deg[b] or (deg[a] == deg[b] and a < b)


def test_determinism():
    a = W.rmat(12, 16, seed=5, whi=255)
    b = W.rmat(12, 16, seed=5, whi=255)
    c = W.rmat(12, 16, seed=6, whi=255)
    assert np.array_equal(a.col, b.col) and np.array_equal(a.w, b.w)
    assert not (a.n == c.n and np.array_equal(a.col, c.col))
    assert np.array_equal(W.uniform_pairs(100, 50, 2), W.uniform_pairs(100, 50, 2))


def test_rmat_structure():
    g = W.rmat(14, 16, seed=18, whi=255)
    check_graph(g, 1, 255)
    assert g.meta["edges_sampled"] == 16 << 14
    assert g.n < (1 << 14)                     # isolated ids dropped by the LCC step
    deg = g.degree()
    assert deg.max() > 50 * np.median(deg)     # heavy-tailed degrees


def test_grid_recipe_small():
    g = W.grid(32, 198, seed=3)                # 2*32*31 = 1984 edges, 10% deleted
    assert g.meta["edges_sampled"] == 1984
    check_graph(g, 500, 1500)
    assert g.m <= 1984 - 198
    rank = W.spt_count_rank(g, 16, seed=3)
    assert sorted(rank.tolist()) == list(range(g.n))


def test_pairs_ranges():
    g, _ = W.load("ba2k")
    p = W.uniform_pairs(g.n, 10000, 2)
    assert p.shape == (10000, 2) and p.max() < g.n
    q = W.degree_pairs(g, 10000, 2)
    deg = g.degree()
    assert deg[q[:, 0]].mean() > 1.5 * deg.mean()  # degree-weighted endpoints


@pytest.mark.parametrize("name", ["rmat18", "grid512"])
def test_inputs_match_stored_digests(name):
    """The generators still produce the inputs whose canonical labelings
    tests/golden/label_digests.json holds (the full-size GPU tests compare
    against those digests)."""
    import importlib.util
    import json
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    spec = importlib.util.spec_from_file_location("make_digests", os.path.join(here, "make_digests.py"))
    md = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(md)
    gold = json.load(open(os.path.join(here, "label_digests.json")))[name]
    g, rank = W.load(name)
    assert md.input_digest(g, rank) == gold["input_sha256"]
