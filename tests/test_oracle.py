"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each pin is chosen so that a plausible mistake in the oracle (a dropped
relaxation, a wrong tie rule, a transposed rank comparison, a missing sort)
fails at least one of them:
  * brute force of the definition on tiny graphs (all-pairs distances from
    scipy, hub of v = highest-ranked vertex of SP_{v,h}; Sec. 1, Lemma 1),
  * closed forms (tree, star, path) and two hand-derived fixtures
    (tests/golden: the "always relax" reading of Algorithm 3 and the
    equal-distance tie rule of the Sec. 5.2 example),
  * the cover property against scipy's Dijkstra (Sec. 1),
  * minimality by DQ_Clean (Algorithm 2, Lemma 2),
  * uniqueness under shuffled root order and randomised tie-breaking,
  * agreement of three independent constructions (definition, Algorithm 3,
    sequential Algorithm 1),
  * structural invariants of a canonical labeling.
"""
import os

import numpy as np
import pytest
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import shortest_path, dijkstra

import oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U32MAX = np.iinfo(np.uint32).max


# ------------------------------------------------------------------ helpers
class G:
    def __init__(self, n, row_ptr, col, w):
        self.n, self.row_ptr, self.col, self.w = n, row_ptr, col, w


def from_edges(n, edges):
    """Symmetric CSR with sorted rows from (a, b, w) undirected edges."""
    adj = [dict() for _ in range(n)]
    for a, b, w in edges:
        assert a != b
        adj[a][b] = w
        adj[b][a] = w
    row = np.zeros(n + 1, np.uint64)
    col, wt = [], []
    for v in range(n):
        for u in sorted(adj[v]):
            col.append(u)
            wt.append(adj[v][u])
        row[v + 1] = len(col)
    return G(n, row, np.array(col, np.uint32), np.array(wt, np.uint32))


def apsp(g):
    A = csr_matrix((g.w.astype(np.float64), g.col.astype(np.int64), g.row_ptr.astype(np.int64)),
                   shape=(g.n, g.n))
    return shortest_path(A, method="D", directed=False)


def brute_chl(g, rank):
    """Definition, written out: (h, d(v,h)) in L_v iff R(h) = max R over SP_{v,h}."""
    D = apsp(g)
    n = g.n
    L = {v: [] for v in range(n)}
    for v in range(n):
        for h in range(n):
            if not np.isfinite(D[v, h]):
                continue
            on_sp = np.where(D[v, :] + D[:, h] == D[v, h])[0]
            if rank[on_sp].max() == rank[h]:
                L[v].append((h, int(D[v, h])))
        L[v].sort(key=lambda t: -int(rank[t[0]]))
    return L


def as_dict(lab):
    return {v: lab.of(v) for v in range(lab.n)}


def random_graph(n, p, wmax, seed, connected=True):
    rng = np.random.default_rng(seed)
    edges = {}
    if connected:
        perm = rng.permutation(n)
        for i in range(1, n):
            a, b = int(perm[i]), int(perm[rng.integers(0, i)])
            edges[(min(a, b), max(a, b))] = int(rng.integers(1, wmax + 1))
    for a in range(n):
        for b in range(a + 1, n):
            if rng.random() < p:
                edges[(a, b)] = int(rng.integers(1, wmax + 1))
    return from_edges(n, [(a, b, w) for (a, b), w in edges.items()])


def read_fixture(name):
    edges, rank, labels, absent = [], {}, [], []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            t = line.split("#")[0].split()
            if not t:
                continue
            if t[0] == "edge":
                edges.append((int(t[1]), int(t[2]), int(t[3])))
            elif t[0] == "rank":
                rank[int(t[1])] = int(t[2])
            elif t[0] == "label":
                labels.append((int(t[1]), int(t[2]), int(t[3])))
            elif t[0] == "absent":
                absent.append((int(t[1]), int(t[2]), int(t[3])))
    n = len(rank)
    r = np.array([rank[v] for v in range(n)], np.uint32)
    return from_edges(n, edges), r, labels, absent


METHODS = ["canonical", "plant", "pll"]


def tiny_cases():
    cases = []
    for s in range(12):
        n = 6 + 3 * s
        for wmax in (1, 2, 9):  # wmax 1 and 2 make many equal-length paths
            g = random_graph(n, 0.15, wmax, seed=100 * s + wmax)
            r = np.random.default_rng(s + 7 * wmax).permutation(n).astype(np.uint32)
            cases.append((f"rand{n}_w{wmax}", g, r))
    # all-equal weights on regular structures: maximal ties
    k = 6
    grid = [(i * k + j, i * k + j + 1, 1) for i in range(k) for j in range(k - 1)]
    grid += [(i * k + j, (i + 1) * k + j, 1) for i in range(k - 1) for j in range(k)]
    cases.append(("grid6", from_edges(k * k, grid), np.random.default_rng(1).permutation(k * k).astype(np.uint32)))
    cases.append(("cycle9", from_edges(9, [(i, (i + 1) % 9, 1) for i in range(9)]),
                  np.random.default_rng(2).permutation(9).astype(np.uint32)))
    cases.append(("k7", from_edges(7, [(a, b, 1) for a in range(7) for b in range(a + 1, 7)]),
                  np.random.default_rng(3).permutation(7).astype(np.uint32)))
    cases.append(("disconnected", from_edges(8, [(0, 1, 2), (1, 2, 2), (3, 4, 1), (5, 6, 3), (6, 7, 3), (5, 7, 6)]),
                  np.random.default_rng(4).permutation(8).astype(np.uint32)))
    return cases


# ------------------------------------------------------------------ P1 brute force
@pytest.mark.parametrize("name,g,rank", tiny_cases(), ids=[c[0] for c in tiny_cases()])
@pytest.mark.parametrize("method", METHODS)
def test_brute_force_definition(name, g, rank, method):
    want = brute_chl(g, rank)
    got = as_dict(O.build_labels(g, rank, method))
    assert got == want


# ------------------------------------------------------------------ hand-derived fixtures
@pytest.mark.parametrize("method", METHODS)
def test_always_relax_reading(method):
    g, rank, labels, _ = read_fixture("a1_counterexample.txt")
    L = O.build_labels(g, rank, method)
    want = {v: [] for v in range(g.n)}
    for v, h, d in labels:
        want[v].append((h, d))
    assert as_dict(L) == want
    assert (0, 10) not in L.of(3)  # the label a pruning reading would emit


@pytest.mark.parametrize("method", METHODS)
def test_equal_distance_tie_rule(method):
    g, rank, _, absent = read_fixture("fig1_tie_fragment.txt")
    L = O.build_labels(g, rank, method)
    for v, h, d in absent:
        assert (h, d) not in L.of(v)
    assert as_dict(L) == brute_chl(g, rank)


# ------------------------------------------------------------------ P2 closed forms
def test_tree_closed_form():
    """On a tree, h is a hub of v iff h has the highest rank on the v-h path."""
    rng = np.random.default_rng(5)
    n = 60
    parent = [None] + [int(rng.integers(0, i)) for i in range(1, n)]
    edges = [(i, parent[i], int(rng.integers(1, 20))) for i in range(1, n)]
    g = from_edges(n, edges)
    rank = rng.permutation(n).astype(np.uint32)

    def path(a, b):
        up = lambda x: [x] + (up(parent[x]) if parent[x] is not None else [])
        pa, pb = up(a), up(b)
        common = next(x for x in pa if x in pb)
        return pa[:pa.index(common) + 1] + pb[:pb.index(common)]

    D = apsp(g)
    for method in METHODS:
        L = O.build_labels(g, rank, method)
        for v in range(n):
            hubs = {h for h, _ in L.of(v)}
            want = {h for h in range(n) if max(rank[path(v, h)]) == rank[h]}
            assert hubs == want
            assert all(d == D[v, h] for h, d in L.of(v))


def test_star_closed_form():
    n = 12
    g = from_edges(n, [(0, i, i) for i in range(1, n)])
    rank = np.array([n - 1] + list(range(n - 1)), np.uint32)  # centre on top
    L = O.build_labels(g, rank, "plant")
    assert L.of(0) == [(0, 0)]
    for i in range(1, n):
        assert L.of(i) == [(0, i), (i, 0)]


def test_path_closed_form():
    """Path with rank increasing toward vertex n-1: every higher-ranked vertex
    toward that end is a hub, at its path distance."""
    n = 10
    w = [3, 1, 4, 1, 5, 9, 2, 6, 5]
    g = from_edges(n, [(i, i + 1, w[i]) for i in range(n - 1)])
    rank = np.arange(n, dtype=np.uint32)
    pre = np.concatenate([[0], np.cumsum(w)])
    for method in METHODS:
        L = O.build_labels(g, rank, method)
        for v in range(n):
            assert L.of(v) == [(h, int(pre[h] - pre[v])) for h in range(n - 1, v - 1, -1)]


# ------------------------------------------------------------------ P3 cover + queries
def test_cover_all_pairs_small():
    g = W.barabasi_albert(300, 3, seed=11)
    rank = W.degree_rank(g)
    L = O.build_labels(g, rank, "plant")
    D = apsp(g)
    u, v = np.meshgrid(np.arange(g.n), np.arange(g.n), indexing="ij")
    pairs = np.stack([u.ravel(), v.ravel()], 1).astype(np.uint32)
    got = O.query(L, rank, pairs, threads=4)
    assert np.array_equal(got, D.ravel().astype(np.uint32))


def test_cover_sampled_pairs_ba2k():
    g, rank = W.load("ba2k")
    L = O.build_labels(g, rank, "plant", threads=4)
    pairs = W.query_pairs(g, 20000, seed=2)
    src = np.unique(pairs[:200, 0])
    A = csr_matrix((g.w.astype(np.float64), g.col.astype(np.int64), g.row_ptr.astype(np.int64)),
                   shape=(g.n, g.n))
    D = dijkstra(A, indices=src)
    sel = np.isin(pairs[:, 0], src)
    p = pairs[sel]
    got = O.query(L, rank, p)
    want = D[np.searchsorted(src, p[:, 0]), p[:, 1]].astype(np.uint32)
    assert np.array_equal(got, want)


def test_query_special_cases():
    g = from_edges(6, [(0, 1, 4), (1, 2, 4), (3, 4, 7), (4, 5, 1)])
    rank = np.array([5, 4, 3, 2, 1, 0], np.uint32)
    L = O.build_labels(g, rank, "canonical")
    q = np.array([[2, 2], [0, 2], [0, 3], [5, 3], [4, 4]], np.uint32)
    assert O.query(L, rank, q).tolist() == [0, 8, U32MAX, 8, 0]


# ------------------------------------------------------------------ P4 minimality
def test_minimality_dq_clean():
    g, rank = W.load("ba2k")
    L = O.build_labels(g, rank, "plant")
    assert O.count_redundant(L, rank) == 0


def test_dq_clean_detects_a_redundant_label():
    """A mistake planted in an oracle output on the CPU must be caught."""
    g, rank = W.load("ba2k")
    L = O.build_labels(g, rank, "plant")
    D = dijkstra(csr_matrix((g.w.astype(np.float64), g.col.astype(np.int64),
                             g.row_ptr.astype(np.int64)), shape=(g.n, g.n)), indices=[5])
    # add (h, d(v,h)) to L_v for a pair whose shortest path holds a better hub
    v = 5
    hubs = {h for h, _ in L.of(v)}
    h = next(int(x) for x in np.argsort(-rank.astype(np.int64))
             if int(x) not in hubs and rank[x] > rank[v] and np.isfinite(D[0, x]))
    lab = L.of(v) + [(h, int(D[0, h]))]
    lab.sort(key=lambda t: -int(rank[t[0]]))
    off = L.offsets.copy()
    off[v + 1:] += 1
    a = int(L.offsets[v])
    hub = np.concatenate([L.hub[:a], [x for x, _ in lab], L.hub[int(L.offsets[v + 1]):]]).astype(np.uint32)
    dist = np.concatenate([L.dist[:a], [d for _, d in lab], L.dist[int(L.offsets[v + 1]):]]).astype(np.uint32)
    bad = O.Labels(off, hub, dist)
    assert O.count_redundant(bad, rank) == 1


# ------------------------------------------------------------------ P5 uniqueness
def test_uniqueness_shuffled_roots_and_ties():
    g = W.barabasi_albert(500, 2, seed=3, wlo=1, whi=3)  # small weights: many ties
    rank = W.degree_rank(g)
    base = O.build_labels(g, rank, "canonical")
    for s in (1, 2, 3):
        roots = np.random.default_rng(s).permutation(g.n).astype(np.uint32)
        for m in ("canonical", "plant"):
            L = O.build_labels(g, rank, m, roots=roots, threads=3, tie_seed=s)
            assert np.array_equal(L.offsets, base.offsets)
            assert np.array_equal(L.hub, base.hub)
            assert np.array_equal(L.dist, base.dist)


# ------------------------------------------------------------------ P6 independent constructions
@pytest.mark.parametrize("which", ["ba2k", "grid24", "rmat10"])
def test_three_constructions_agree(which):
    if which == "ba2k":
        g, rank = W.load("ba2k")
    elif which == "grid24":
        g = W.grid(24, 55, seed=9)
        rank = W.spt_count_rank(g, 16, seed=9)
    else:
        g = W.rmat(10, 8, seed=10, wlo=1, whi=20)
        rank = W.degree_rank(g)
    a = O.build_labels(g, rank, "canonical", threads=4)
    b = O.build_labels(g, rank, "plant", threads=4)
    c = O.build_labels(g, rank, "pll")
    for x in (b, c):
        assert np.array_equal(a.offsets, x.offsets)
        assert np.array_equal(a.hub, x.hub)
        assert np.array_equal(a.dist, x.dist)


# ------------------------------------------------------------------ P7 invariants
def test_invariants():
    g, rank = W.load("ba2k")
    L = O.build_labels(g, rank, "plant")
    top = int(np.argmax(rank))
    D = dijkstra(csr_matrix((g.w.astype(np.float64), g.col.astype(np.int64),
                             g.row_ptr.astype(np.int64)), shape=(g.n, g.n)), indices=[top])[0]
    for v in range(g.n):
        lab = L.of(v)
        assert lab[-1] == (v, 0)                       # self label last
        assert lab[0] == (top, int(D[v]))              # global top vertex first (connected)
        r = [int(rank[h]) for h, _ in lab]
        assert r == sorted(r, reverse=True) and len(set(r)) == len(r)
        assert min(r) == int(rank[v])                  # every hub ranks at least R(v)


def test_subset_of_roots_is_hub_partition():
    """Trees are independent (Sec. 5.2): labels of a root subset are exactly the
    full labels whose hub lies in that subset."""
    g, rank = W.load("ba2k")
    full = O.build_labels(g, rank, "plant")
    roots = np.arange(0, g.n, 7, dtype=np.uint32)
    part = O.build_labels(g, rank, "plant", roots=roots)
    keep = np.isin(full.hub, roots)
    assert np.array_equal(part.hub, full.hub[keep])
    assert np.array_equal(part.dist, full.dist[keep])


def test_stats_psi():
    g, rank = W.load("ba2k")
    L, st = O.build_labels(g, rank, "plant", with_stats=True)
    assert int(st[:, 2].sum()) == L.total
    assert (st[:, 0] >= st[:, 2]).all()              # labels <= settled per tree
    Lc, stc = O.build_labels(g, rank, "canonical", with_stats=True)
    assert (stc[:, 0] == g.n).all()                   # the definition settles everything
    assert st[:, 0].sum() < stc[:, 0].sum()           # early termination explores less


def test_pll_query_entry_count():
    """The label entries Algorithm 1's distance queries read (a work count of
    the bench's roofline). The first tree reads none (no labels exist yet). In
    the second tree every list holds exactly the top hub's label, so the count
    is the root's one entry plus one per settled vertex that the rank query
    does not drop, which is every settled vertex but the root (the top vertex
    outranks the root and is dropped). Later trees read at least the root's
    list."""
    g, rank = W.load("ba2k")
    L, st = O.build_labels(g, rank, "pll", with_stats=True)
    assert L.total == O.build_labels(g, rank, "plant").total
    q, settled = st[:, 3].astype(np.int64), st[:, 0].astype(np.int64)
    assert q[0] == 0
    assert q[1] == 1 + (settled[1] - 2) + 1  # root list + non-root, non-top vertices + the root's own query
    assert (q[1:] >= 1).all()
    assert (st[:, 2] <= st[:, 0]).all()


def test_overflow_flag():
    big = 2 ** 31
    g = from_edges(4, [(0, 1, big), (1, 2, big), (2, 3, 5)])
    rank = np.array([3, 2, 1, 0], np.uint32)
    assert O.build_labels(g, rank, "plant").overflow
    assert not O.build_labels(from_edges(3, [(0, 1, 5), (1, 2, 5)]), rank[:3] - 1, "plant").overflow


# ------------------------------------------------------------------ phased labeling (Hybrid, Sec. 5.2/5.3)
def phase_schedules(n):
    """phase ends by rank position: one phase (Algorithm 3), the top root
    alone first, every root its own phase, and irregular splits"""
    out = [[n], [1, n], list(range(1, n + 1))]
    out.append(sorted({min(n, x) for x in (2, 3, 5, 8, 13, n)}))
    out.append(sorted({max(1, n // 3), max(1, 2 * n // 3), n}))
    return [list(e) for e in {tuple(e) for e in out}]


@pytest.mark.parametrize("name,g,rank", tiny_cases(), ids=[c[0] for c in tiny_cases()])
def test_phased_brute_force(name, g, rank):
    """Pruning each phase's trees by every label of the earlier phases (a
    rank-closed hub set) gives the canonical labeling for every schedule."""
    want = brute_chl(g, rank)
    for ends in phase_schedules(g.n):
        assert as_dict(O.build_labels_phased(g, rank, ends)) == want, ends


@pytest.mark.parametrize("which", ["ba2k", "grid24", "rmat10"])
def test_phased_agrees_and_prunes(which):
    """Equal to Algorithm 3 on larger graphs under seeded random schedules;
    with every root its own phase the trees relax exactly the arcs sequential
    Algorithm 1 relaxes (the same pruning, query for query), and any split
    relaxes fewer arcs than the single phase."""
    if which == "ba2k":
        g, rank = W.load("ba2k")
    elif which == "grid24":
        g = W.grid(24, 60, seed=24)
        rank = W.spt_count_rank(g, 16, seed=24)
    else:
        g = W.rmat(10, 8, seed=10, wlo=1, whi=50)
        rank = W.degree_rank(g)
    ref = O.build_labels(g, rank, "plant")
    _, st1 = O.build_labels_phased(g, rank, [g.n], with_stats=True)
    rng = np.random.default_rng(5)
    for _ in range(3):
        k = int(rng.integers(2, 12))
        ends = sorted(set(rng.integers(1, g.n, size=k).tolist()) | {g.n})
        L, st = O.build_labels_phased(g, rank, ends, threads=4, with_stats=True)
        assert np.array_equal(L.offsets, ref.offsets) and np.array_equal(L.hub, ref.hub)
        assert np.array_equal(L.dist, ref.dist)
        assert st[:, 1].sum() < st1[:, 1].sum()
    _, st_each = O.build_labels_phased(g, rank, np.arange(1, g.n + 1), with_stats=True)
    _, st_pll = O.build_labels(g, rank, "pll", with_stats=True)
    assert st_each[:, 1].sum() == st_pll[:, 1].sum()


# ------------------------------------------------------------------ Common Label Table (Sec. 5.3)
@pytest.mark.parametrize("name,g,rank", tiny_cases(), ids=[c[0] for c in tiny_cases()])
@pytest.mark.parametrize("eta", [1, 2, 5])
def test_common_label_table_brute_force(name, g, rank, eta):
    """Pruning the trees with distance queries on the labels of the eta most
    important hubs leaves the labeling equal to the definition."""
    got = as_dict(O.build_labels(g, rank, "plant_clt", eta=eta))
    assert got == brute_chl(g, rank)


@pytest.mark.parametrize("eta", [1, 3])
def test_common_label_table_fixtures(eta):
    for fx in ("a1_counterexample.txt", "fig1_tie_fragment.txt"):
        g, rank, _, _ = read_fixture(fx)
        assert as_dict(O.build_labels(g, rank, "plant_clt", eta=eta)) == brute_chl(g, rank)


@pytest.mark.parametrize("which", ["ba2k", "grid24", "rmat10"])
@pytest.mark.parametrize("eta", [3, 16])
def test_common_label_table_agrees_and_prunes(which, eta):
    if which == "ba2k":
        g, rank = W.load("ba2k")
    elif which == "grid24":
        g = W.grid(24, 55, seed=9)
        rank = W.spt_count_rank(g, 16, seed=9)
    else:
        g = W.rmat(10, 8, seed=10, wlo=1, whi=20)
        rank = W.degree_rank(g)
    a, sa = O.build_labels(g, rank, "plant", threads=4, with_stats=True)
    b, sb = O.build_labels(g, rank, "plant_clt", threads=4, eta=eta, with_stats=True)
    assert np.array_equal(a.offsets, b.offsets)
    assert np.array_equal(a.hub, b.hub)
    assert np.array_equal(a.dist, b.dist)
    assert (sb[:, 2] == sa[:, 2]).all()                  # labels per tree unchanged
    n = g.n
    pos = n - 1 - rank.astype(np.int64)
    order = np.argsort(pos)
    top = pos[order] < eta
    assert (sb[top] == sa[top]).all()                    # top trees are not pruned
    assert sb[:, 1].sum() < sa[:, 1].sum()               # the others scan fewer arcs


def test_common_label_table_root_subset():
    """Trees of roots outside the table still see the whole table."""
    g, rank = W.load("ba2k")
    full = O.build_labels(g, rank, "plant")
    n = g.n
    order = np.empty(n, np.uint32)
    order[n - 1 - rank.astype(np.int64)] = np.arange(n, dtype=np.uint32)
    for roots in (order[100:400], order[10:30], order[::9]):
        part = O.build_labels(g, rank, "plant_clt", roots=roots, eta=16, threads=2)
        keep = np.isin(full.hub, roots)
        assert np.array_equal(part.hub, full.hub[keep])
        assert np.array_equal(part.dist, full.dist[keep])


# ------------------------------------------------------------------ shortest-path recovery (Sec. 5.4, Extensions)
def brute_parent(g, rank, D, v, h, d):
    """Highest-ranked neighbour p of v with D[h, p] + w(p, v) = d, from the
    all-pairs distances (no labels involved)."""
    best = None
    for e in range(int(g.row_ptr[v]), int(g.row_ptr[v + 1])):
        p = int(g.col[e])
        if D[h, p] + int(g.w[e]) == d and (best is None or rank[p] > rank[best]):
            best = p
    return best


@pytest.mark.parametrize("name,g,rank", tiny_cases()[::3], ids=[c[0] for c in tiny_cases()[::3]])
def test_parents_brute_force(name, g, rank):
    D = apsp(g)
    L = O.build_labels(g, rank, "canonical")
    par = O.parents(g, rank, L)
    for v in range(g.n):
        for k in range(int(L.offsets[v]), int(L.offsets[v + 1])):
            h, d = int(L.hub[k]), int(L.dist[k])
            want = v if h == v else brute_parent(g, rank, D, v, h, d)
            assert int(par[k]) == want, (v, h)


@pytest.mark.parametrize("name,g,rank", tiny_cases()[::3], ids=[c[0] for c in tiny_cases()[::3]])
def test_paths_are_canonical_shortest_paths(name, g, rank):
    """Every recovered path is a walk over edges of total weight D[u, v] that
    passes the highest-ranked vertex of SP_{u,v}; disconnected pairs give []."""
    D = apsp(g)
    n = g.n
    L = O.build_labels(g, rank, "plant")
    par = O.parents(g, rank, L)
    wt = {}
    for v in range(n):
        for e in range(int(g.row_ptr[v]), int(g.row_ptr[v + 1])):
            wt[(v, int(g.col[e]))] = int(g.w[e])
    pairs = [(u, v) for u in range(n) for v in range(n)]
    for (u, v), path in zip(pairs, O.paths(L, rank, par, pairs)):
        if not np.isfinite(D[u, v]):
            assert path == []
            continue
        assert path[0] == u and path[-1] == v
        assert sum(wt[(a, b)] for a, b in zip(path, path[1:])) == D[u, v]
        on_sp = np.where(D[u, :] + D[:, v] == D[u, v])[0]
        top = int(on_sp[np.argmax(rank[on_sp])])
        assert top in path


# ------------------------------------------------------------------ closed form: K_{2,m}
def double_star_closed_form(g, rank):
    """Labels of W.double_star by hand: c (vertex 0, lowest rank) reaches each
    leaf l directly at w_l, and no other vertex lies on that edge, so l is its
    hub; t (top rank) lies on every other shortest path (each leaf-to-leaf path
    through c has a twin of equal length through t), so it is the only other
    hub anywhere. L_c = t at 2 min(w), the leaves by rank descending, c; L_t =
    t; L_l = t at w_l, l."""
    m = g.n - 2
    w = g.w[:m].astype(np.uint64)  # c's row: leaves 2..m+1 in order
    leaves = np.arange(2, g.n)
    by_rank = leaves[np.argsort(-rank[leaves].astype(np.int64), kind="stable")]
    off = [0, m + 2, m + 3]
    hub = [1, *by_rank, 0, 1]
    dist = [2 * int(w.min()), *[int(w[l - 2]) for l in by_rank], 0, 0]
    for l in leaves:
        off.append(off[-1] + 2)
        hub += [1, int(l)]
        dist += [int(w[l - 2]), 0]
    return np.array(off, np.uint64), np.array(hub, np.uint32), np.array(dist, np.uint32)


@pytest.mark.parametrize("m,seed", [(1, 1), (7, 2), (300, 3)])
def test_double_star_closed_form(m, seed):
    g, rank = W.double_star(m, seed)
    off, hub, dist = double_star_closed_form(g, rank)
    for method in ("canonical", "plant", "pll"):
        L = O.build_labels(g, rank, method)
        assert np.array_equal(L.offsets, off) and np.array_equal(L.hub, hub), method
        assert np.array_equal(L.dist, dist), method


def test_phased_root_prefix_is_hub_partition():
    """A phased build that stops after the top R roots gives exactly the
    canonical labels whose hub ranks among the top R (trees are independent,
    Sec. 5.2), whatever the schedule before R."""
    g, rank = W.load("ba2k")
    full = O.build_labels(g, rank, "canonical")
    pos = g.n - 1 - rank.astype(np.int64)
    for ends in ([37], [8, 16, 37], [1, 2, 3, 500], [304, 608, 1216, 1999]):
        part = O.build_labels_phased(g, rank, ends, threads=3)
        keep = pos[full.hub] < ends[-1]
        assert np.array_equal(part.hub, full.hub[keep]), ends
        assert np.array_equal(part.dist, full.dist[keep]), ends
        cnt = np.add.reduceat(keep.astype(np.int64), full.offsets[:-1].astype(np.int64)) if full.total else 0
        assert np.array_equal(np.diff(part.offsets.astype(np.int64)), np.where(np.diff(full.offsets.astype(np.int64)) > 0, cnt, 0)), ends
