"""Seeded synthetic workloads for canonical hub labeling.

Input synthesis only: graphs, ranking functions and query pairs. Nothing here
computes any part of the labeling method; the CPU oracle (``oracle``) and the
GPU library (``paper_1907_00140_gb300``) both consume these arrays.

The graph families stand in for the paper's datasets (Sec. 7.1, Table 2):
R-MAT and Barabasi-Albert graphs with degree ranking for the scale-free
networks, a 2-D grid with a sampled shortest-path-tree ranking for the road
networks (betweenness approximated by sampling trees, Sec. 7.1).

The generators are plain C (``chl_gen.c``), built with gcc on first use.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "chl_gen.c")
_LIB = os.path.join(_HERE, "libchlgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile chl_gen.c into libchlgen.so (in-tree) if missing or stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Graph(C.Structure):
    _fields_ = [("n", C.c_uint32), ("m", C.c_uint64),
                ("row_ptr", C.POINTER(C.c_uint64)), ("col", C.POINTER(C.c_uint32)),
                ("w", C.POINTER(C.c_uint32)), ("n_before", C.c_uint32),
                ("m_sampled", C.c_uint64)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P, u32, u64, d = C.POINTER, C.c_uint32, C.c_uint64, C.c_double
            lib.gen_ba.argtypes = [u32, u32, u64, u32, u32, P(_Graph)]
            lib.gen_rmat.argtypes = [u32, u32, d, d, d, u64, u32, u32, P(_Graph)]
            lib.gen_grid.argtypes = [u32, u64, u64, P(_Graph)]
            lib.gen_graph_free.argtypes = [P(_Graph)]
            lib.gen_degree_rank.argtypes = [u32, C.c_void_p, C.c_void_p]
            lib.gen_spt_count_rank.argtypes = [u32, C.c_void_p, C.c_void_p, C.c_void_p, u32, u64,
                                               C.c_void_p]
            lib.gen_uniform_pairs.argtypes = [u32, u64, u64, C.c_void_p]
            lib.gen_degree_pairs.argtypes = [u32, C.c_void_p, u64, u64, C.c_void_p]
            lib.gen_unit_doubles.argtypes = [u64, u64, u64, C.c_void_p]
            _lib = lib
    return _lib


@dataclass
class Graph:
    """Undirected weighted graph as a symmetric CSR (every edge stored as two arcs)."""
    n: int
    row_ptr: np.ndarray  # uint64 [n+1]
    col: np.ndarray      # uint32 [2m], each row sorted by neighbour id
    w: np.ndarray        # uint32 [2m], >= 1
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def num_arcs(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def m(self) -> int:
        return self.num_arcs // 2

    def degree(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int64)

    def edges(self):
        """(u, v, w) arrays of the undirected edges with u < v."""
        src = np.repeat(np.arange(self.n, dtype=np.uint32), np.diff(self.row_ptr.astype(np.int64)))
        keep = src < self.col
        return src[keep], self.col[keep], self.w[keep]


def _take(g: _Graph, name: str, **meta) -> Graph:
    lib = _load()
    n, arcs = g.n, 2 * g.m
    row = np.ctypeslib.as_array(g.row_ptr, shape=(n + 1,)).copy()
    col = np.ctypeslib.as_array(g.col, shape=(arcs,)).copy() if arcs else np.zeros(0, np.uint32)
    w = np.ctypeslib.as_array(g.w, shape=(arcs,)).copy() if arcs else np.zeros(0, np.uint32)
    meta.update(n_ids=int(g.n_before), edges_sampled=int(g.m_sampled))
    lib.gen_graph_free(C.byref(g))
    return Graph(int(n), row, col, w, name, meta)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"{what} failed with code {rc}")


def barabasi_albert(n: int, m: int, seed: int, wlo: int = 1, whi: int = 100) -> Graph:
    """Clique on m+1 vertices, then each new vertex joins m distinct vertices
    drawn proportionally to degree; weights uniform in [wlo, whi]."""
    g = _Graph()
    _check(_load().gen_ba(n, m, seed, wlo, whi, C.byref(g)), "gen_ba")
    return _take(g, f"ba_n{n}_m{m}", seed=seed, wlo=wlo, whi=whi)


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 0, wlo: int = 1, whi: int = 255) -> Graph:
    """R-MAT, symmetrised, self-loops and duplicates dropped, largest component
    kept (relabelled in id order); weights uniform in [wlo, whi]."""
    g = _Graph()
    _check(_load().gen_rmat(scale, edge_factor, a, b, c, seed, wlo, whi, C.byref(g)), "gen_rmat")
    return _take(g, f"rmat{scale}", seed=seed, wlo=wlo, whi=whi)


def grid(side: int, n_delete: int, seed: int) -> Graph:
    """side x side 4-neighbour grid, n_delete edges removed uniformly without
    replacement, largest component kept; weights llround(1000*U[0.5,1.5))."""
    g = _Graph()
    _check(_load().gen_grid(side, n_delete, seed, C.byref(g)), "gen_grid")
    return _take(g, f"grid{side}", seed=seed, n_delete=n_delete)


def degree_rank(g: Graph) -> np.ndarray:
    """R(v): degree descending, ties by smaller id first; larger R = more important."""
    r = np.empty(g.n, np.uint32)
    _check(_load().gen_degree_rank(g.n, g.row_ptr.ctypes.data, r.ctypes.data), "gen_degree_rank")
    return r


def spt_count_rank(g: Graph, samples: int = 256, seed: int = 0) -> np.ndarray:
    """R(v) by the number of sampled shortest-path-tree paths through v
    (parent = tight predecessor of smallest id), descending, ties by id."""
    r = np.empty(g.n, np.uint32)
    _check(_load().gen_spt_count_rank(g.n, g.row_ptr.ctypes.data, g.col.ctypes.data,
                                      g.w.ctypes.data, samples, seed, r.ctypes.data),
           "gen_spt_count_rank")
    return r


def uniform_pairs(n: int, q: int, seed: int) -> np.ndarray:
    """q query pairs, endpoints i.i.d. uniform over [0, n); shape (q, 2) uint32."""
    p = np.empty((q, 2), np.uint32)
    _check(_load().gen_uniform_pairs(n, q, seed, p.ctypes.data), "gen_uniform_pairs")
    return p


def degree_pairs(g: Graph, q: int, seed: int) -> np.ndarray:
    """q query pairs, both endpoints drawn proportionally to degree."""
    p = np.empty((q, 2), np.uint32)
    _check(_load().gen_degree_pairs(g.n, g.row_ptr.ctypes.data, q, seed, p.ctypes.data),
           "gen_degree_pairs")
    return p


def unit_doubles(count: int, seed: int, stream: int = 0) -> np.ndarray:
    """count uniform doubles in [0, 1) from an independent seeded stream."""
    out = np.empty(count, np.float64)
    _check(_load().gen_unit_doubles(count, seed, stream, out.ctypes.data), "gen_unit_doubles")
    return out


def double_star(m: int, seed: int) -> tuple:
    """K_{2,m} with its ranking: vertex 0 (c, lowest rank) and vertex 1 (t,
    highest rank) are both joined to the m leaves 2..m+1, and leaf l's two
    edges carry the same weight U{1..100}, so every leaf-to-leaf shortest path
    has a twin through t. The leaves' ranks are a seeded permutation of
    [1, m]. Under this ranking c is the one vertex with a label list of length
    m + 2 (every leaf, t and itself); the whole labeling has about 3m labels.
    Returns (graph, rank)."""
    n = m + 2
    w = (1 + np.floor(unit_doubles(m, seed, 0) * 100)).astype(np.uint32)
    perm = np.argsort(unit_doubles(m, seed, 1), kind="stable").astype(np.uint32)
    deg = np.concatenate([[m, m], np.full(m, 2)]).astype(np.uint64)
    row = np.concatenate([[0], np.cumsum(deg)]).astype(np.uint64)
    col = np.empty(int(row[-1]), np.uint32)
    ww = np.empty(int(row[-1]), np.uint32)
    leaves = np.arange(2, n, dtype=np.uint32)
    col[0:m], ww[0:m] = leaves, w          # c's row
    col[m:2 * m], ww[m:2 * m] = leaves, w  # t's row
    col[2 * m::2], col[2 * m + 1::2] = 0, 1  # each leaf: c, then t
    ww[2 * m::2], ww[2 * m + 1::2] = w, w
    rank = np.empty(n, np.uint32)
    rank[0], rank[1] = 0, n - 1
    rank[2:] = 1 + perm
    return Graph(n, row, col, ww, f"double_star_m{m}", {"seed": seed}), rank


# ---------------------------------------------------------------- named workloads
# The five workloads of the benchmark plan. Each returns (graph, rank).

def ba2k():
    """Barabasi-Albert n=2,000, m=3, weights U{1..100}, degree rank (seed 1)."""
    g = barabasi_albert(2000, 3, seed=1, wlo=1, whi=100)
    return g, degree_rank(g)


def rmat18():
    """R-MAT scale 18, edge factor 16, a=.57 b=c=.19, weights U{1..255}, degree rank (seed 18)."""
    g = rmat(18, 16, 0.57, 0.19, 0.19, seed=18, wlo=1, whi=255)
    return g, degree_rank(g)


def grid512():
    """512x512 grid, 52,326 of 523,264 edges deleted, weights llround(1000*U[.5,1.5)),
    rank by paths through v in 256 sampled shortest-path trees (seed 512)."""
    g = grid(512, 52326, seed=512)
    return g, spt_count_rank(g, 256, seed=512)


def rmat21():
    """R-MAT scale 21, edge factor 16, a=.57 b=c=.19, weights U{1..1000}, degree rank (seed 21)."""
    g = rmat(21, 16, 0.57, 0.19, 0.19, seed=21, wlo=1, whi=1000)
    return g, degree_rank(g)


def serving_ba(i: int):
    """The i-th (0..7) Barabasi-Albert build request of the serving workload."""
    ns = [10_000, 25_000, 50_000, 75_000, 100_000, 125_000, 150_000, 200_000]
    ms = [3, 4, 5, 6, 7, 8, 3, 8]
    g = barabasi_albert(ns[i], ms[i], seed=100 + i, wlo=1, whi=100)
    return g, degree_rank(g)


WORKLOADS = {"ba2k": ba2k, "rmat18": rmat18, "grid512": grid512, "rmat21": rmat21}


def load(name: str):
    """(graph, rank) of a named workload; graph.name is set to `name`."""
    g, r = WORKLOADS[name]()
    g.name = name
    return g, r


def query_pairs(name_or_n, q: int = 100_000, seed: int = 2) -> np.ndarray:
    n = name_or_n if isinstance(name_or_n, int) else name_or_n.n
    return uniform_pairs(n, q, seed)
