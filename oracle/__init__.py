"""CPU oracle for canonical hub labeling — TEST INFRASTRUCTURE ONLY.

Plain restatement of the paper's definitions in C (``chl_oracle.c``), built with
gcc on first use. Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the GPU library
(``paper_1907_00140_gb300``) never does, and the two share no code.

Functions follow the paper:
  * ``build_labels``: the canonical labeling (Sec. 1), three independent ways:
      ``"canonical"`` — the definition (h is a hub of v iff h is the
      highest-ranked vertex of SP_{v,h}; Sec. 1, Lemma 1 in Sec. 4.1);
      ``"plant"`` — Algorithm 3 (PLaNTDijkstra) with early termination;
      ``"pll"`` — Algorithm 1 run sequentially in rank order (Sec. 4).
  * ``query``: PPSD by linear merge of rank-sorted lists (Sec. 1, Sec. 6 QLSN).
  * ``count_redundant``: labels that ``DQ_Clean`` (Algorithm 2) flags.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "chl_oracle.c")
_LIB = os.path.join(_HERE, "libchloracle.so")
_lock = threading.Lock()
_lib = None

METHODS = {"canonical": 0, "plant": 1, "pll": 2, "plant_clt": 3}


def build(force: bool = False) -> str:
    """Compile chl_oracle.c into liborc (in-tree) if missing or stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lpthread"],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Labels(C.Structure):
    _fields_ = [("offsets", C.POINTER(C.c_uint64)), ("hub", C.POINTER(C.c_uint32)),
                ("dist", C.POINTER(C.c_uint32)), ("total", C.c_uint64), ("overflow", C.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            vp, u32, u64, i32 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int
            lib.orc_build.argtypes = [u32, vp, vp, vp, vp, i32, vp, u64, i32, u64, u32,
                                      C.POINTER(_Labels), vp]
            lib.orc_build_phased.argtypes = [u32, vp, vp, vp, vp, vp, u32, i32,
                                             C.POINTER(_Labels), vp]
            lib.orc_labels_free.argtypes = [C.POINTER(_Labels)]
            lib.orc_query.argtypes = [u32, vp, vp, vp, vp, vp, u64, vp, i32]
            lib.orc_count_redundant.argtypes = [u32, vp, vp, vp, vp]
            lib.orc_count_redundant.restype = u64
            _lib = lib
    return _lib


@dataclass
class Labels:
    """Per-vertex labels: L_v = (hub, dist)[offsets[v]:offsets[v+1]], hubs in
    descending rank."""
    offsets: np.ndarray  # uint64 [n+1]
    hub: np.ndarray      # uint32 [T]
    dist: np.ndarray     # uint32 [T]
    overflow: bool = False

    @property
    def n(self) -> int:
        return len(self.offsets) - 1

    @property
    def total(self) -> int:
        return int(self.offsets[-1])

    def of(self, v: int):
        a, b = int(self.offsets[v]), int(self.offsets[v + 1])
        return list(zip(self.hub[a:b].tolist(), self.dist[a:b].tolist()))


def _u(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def build_labels(g, rank, method: str = "plant", roots=None, threads: int = 1,
                 tie_seed: int = 0, with_stats: bool = False, eta: int = 16):
    """Canonical labels of graph `g` (workloads.Graph or any object with n,
    row_ptr, col, w) under ranking `rank`.

    method: "canonical" (the definition), "plant" (Algorithm 3), "pll"
    (sequential Algorithm 1) or "plant_clt" (Algorithm 3 pruned by the Common
    Label Table of the `eta` most important hubs, Sec. 5.3; eta is capped at n).

    roots: None = every vertex in descending rank; else only labels with hub
    in `roots` are produced (each tree is independent, Sec. 5.2).
    tie_seed != 0 randomises the pop order of equal-distance vertices.
    Returns Labels, or (Labels, stats[k,4] = settled, arcs scanned, labels per
    root, label entries read by the distance queries (Algorithm 1 only; the
    phased method also counts them)) when with_stats.
    """
    lib = _load()
    n = int(g.n)
    row, col, w = _u(g.row_ptr, np.uint64), _u(g.col, np.uint32), _u(g.w, np.uint32)
    rank = _u(rank, np.uint32)
    if roots is None:
        rarr, nroots, rptr = None, n, None
    else:
        rarr = _u(roots, np.uint32)
        nroots, rptr = len(rarr), rarr.ctypes.data
    stats = np.zeros((nroots, 4), np.uint64) if with_stats else None
    out = _Labels()
    rc = lib.orc_build(n, row.ctypes.data, col.ctypes.data, w.ctypes.data, rank.ctypes.data,
                       METHODS[method], rptr, nroots if rarr is not None else 0,
                       int(threads), int(tie_seed), min(int(eta), n), C.byref(out),
                       stats.ctypes.data if stats is not None else None)
    if rc != 0:
        raise RuntimeError(f"orc_build failed: {rc}")
    try:
        T = int(out.total)
        off = np.ctypeslib.as_array(out.offsets, shape=(n + 1,)).copy()
        hub = np.ctypeslib.as_array(out.hub, shape=(T,)).copy() if T else np.zeros(0, np.uint32)
        dist = np.ctypeslib.as_array(out.dist, shape=(T,)).copy() if T else np.zeros(0, np.uint32)
        L = Labels(off, hub, dist, bool(out.overflow))
    finally:
        lib.orc_labels_free(C.byref(out))
    return (L, stats) if with_stats else L


def build_labels_phased(g, rank, ends, threads: int = 1, with_stats: bool = False):
    """Labels built in phases, the Hybrid of Sec. 5.2 as label-pruned phases:
    phase k holds the roots of rank positions [ends[k-1], ends[k]) (ends
    increasing, last <= n); its trees run Algorithm 3 and also skip a popped
    vertex whose distance query over every label of the earlier phases' roots
    is at most its distance (hubs ranked above all of the phase's roots, the
    condition of Sec. 5.3). The result must be the canonical labeling, or with
    a last end below n its labels whose hub is among the top ends[-1] (trees
    are independent, Sec. 5.2).
    Returns Labels, or (Labels, stats[n,4] by rank position) when with_stats."""
    lib = _load()
    n = int(g.n)
    row, col, w = _u(g.row_ptr, np.uint64), _u(g.col, np.uint32), _u(g.w, np.uint32)
    rank = _u(rank, np.uint32)
    ends = _u(np.asarray(ends), np.uint32)
    stats = np.zeros((n, 4), np.uint64) if with_stats else None
    out = _Labels()
    rc = lib.orc_build_phased(n, row.ctypes.data, col.ctypes.data, w.ctypes.data, rank.ctypes.data,
                              ends.ctypes.data, len(ends), int(threads), C.byref(out),
                              stats.ctypes.data if stats is not None else None)
    if rc != 0:
        raise RuntimeError(f"orc_build_phased failed: {rc}")
    try:
        T = int(out.total)
        off = np.ctypeslib.as_array(out.offsets, shape=(n + 1,)).copy()
        hub = np.ctypeslib.as_array(out.hub, shape=(T,)).copy() if T else np.zeros(0, np.uint32)
        dist = np.ctypeslib.as_array(out.dist, shape=(T,)).copy() if T else np.zeros(0, np.uint32)
        L = Labels(off, hub, dist, bool(out.overflow))
    finally:
        lib.orc_labels_free(C.byref(out))
    return (L, stats) if with_stats else L


def query(L: Labels, rank, pairs, threads: int = 1) -> np.ndarray:
    """d(u,v) for each pair; UINT32_MAX where u and v share no hub."""
    lib = _load()
    pairs = _u(pairs, np.uint32).reshape(-1, 2)
    out = np.empty(len(pairs), np.uint32)
    rank = _u(rank, np.uint32)
    rc = lib.orc_query(L.n, L.offsets.ctypes.data, L.hub.ctypes.data, L.dist.ctypes.data,
                       rank.ctypes.data, pairs.ctypes.data, len(pairs), out.ctypes.data,
                       int(threads))
    if rc != 0:
        raise ValueError(f"orc_query failed: {rc}")
    return out


def count_redundant(L: Labels, rank) -> int:
    """Number of labels that DQ_Clean (Algorithm 2) would delete."""
    lib = _load()
    rank = _u(rank, np.uint32)
    return int(lib.orc_count_redundant(L.n, L.offsets.ctypes.data, L.hub.ctypes.data,
                                       L.dist.ctypes.data, rank.ctypes.data))


# ------------------------------------------------------------------ shortest-path recovery
def parents(g, rank, L: Labels) -> np.ndarray:
    """SPT parent of every label, aligned with L.hub/L.dist (Sec. 5.4,
    Extensions: the parent of v in the tree of h stored with the label).
    For (h, d) in L_v, v != h: the highest-ranked neighbour p of v on a shortest
    h-v path, i.e. with d(h, p) + w(p, v) = d. Every vertex of those paths has h
    as a hub (h ranks highest on SP_{v,h}, hence on each sub-path), so d(h, p)
    is read from p's own labels. For v = h the parent is h."""
    n = int(g.n)
    row = np.asarray(g.row_ptr, np.int64)
    col = np.asarray(g.col)
    w = np.asarray(g.w)
    dist_of = [dict(zip(L.hub[L.offsets[v]:L.offsets[v + 1]].tolist(),
                        L.dist[L.offsets[v]:L.offsets[v + 1]].tolist())) for v in range(n)]
    out = np.empty(L.total, np.uint32)
    for v in range(n):
        for k in range(int(L.offsets[v]), int(L.offsets[v + 1])):
            h, d = int(L.hub[k]), int(L.dist[k])
            if h == v:
                out[k] = v
                continue
            best = None
            for e in range(row[v], row[v + 1]):
                p = int(col[e])
                dp = dist_of[p].get(h)
                if dp is not None and dp + int(w[e]) == d and (best is None or rank[p] > rank[best]):
                    best = p
            out[k] = best
    return out


def paths(L: Labels, rank, par: np.ndarray, pairs) -> list:
    """Shortest u-v path for each pair (list of vertex lists; [] when u and v
    share no hub): the canonical hub H of the pair (minimum d(u,h) + d(v,h),
    then the highest rank), then parents from u up to H and from v up to H."""
    res = []
    for u, v in np.asarray(pairs).tolist():
        Lu = dict(zip(L.hub[L.offsets[u]:L.offsets[u + 1]].tolist(),
                      range(int(L.offsets[u]), int(L.offsets[u + 1]))))
        best = None
        for k in range(int(L.offsets[v]), int(L.offsets[v + 1])):
            h = int(L.hub[k])
            if h in Lu:
                key = (int(L.dist[Lu[h]]) + int(L.dist[k]), -int(rank[h]))
                if best is None or key < best[0]:
                    best = (key, h)
        if best is None:
            res.append([])
            continue
        H = best[1]

        def up(x):
            walk = [x]
            while x != H:
                a, b = int(L.offsets[x]), int(L.offsets[x + 1])
                k = a + int(np.nonzero(L.hub[a:b] == H)[0][0])
                x = int(par[k])
                walk.append(x)
            return walk
        a, b = up(u), up(v)
        res.append(a + b[::-1][1:])
    return res
