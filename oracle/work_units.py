"""Algorithmic work units of each benchmark workload, computed by the oracle.

TEST/BENCH INFRASTRUCTURE: calls only ``oracle`` and ``workloads``.

For the PLaNT build (Algorithm 3 with early termination, Sec. 5.2) the units
are, summed over all roots h:
  S = vertices settled (popped) by the tree of h,
  A = arcs scanned by those vertices,
  T = labels emitted (= total size of the canonical labeling).
T is exact up to `pll_below` vertices: sequential Algorithm 1 (pruned
Dijkstra with rank queries, Sec. 4) builds the same labeling quickly; above
that it is estimated like S and A. S and A are exact for small workloads and
otherwise a stratified estimate: every one of the 64 most important roots,
then rank-position strata of doubling width with `per_stratum` seeded roots
each (mean x stratum size), with a standard error.

With the Common Label Table (Sec. 5.3) the trees explore less; the entry
"<workload>/clt<eta>" holds S and A of Algorithm 3 pruned by the table of the
eta most important hubs (the table's own trees included), same sampling.

The entry "<workload>/pll" holds S and A of sequential Algorithm 1 (every
tree pruned by distance queries over all labels of the hubs ranked above its
root): the work floor of the label-pruned (hybrid) build, exact; Q counts the
label entries its distance queries read (the root's list once per tree, then
the settled vertex's list up to the first witness).

Usage:  python oracle/work_units.py [workload[/clt<eta>|/pll] ...]   (writes oracle/work_units.json)
"""
import json
import os
import sys
import time

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "work_units.json")


def strata(n):
    edges = [0, 64]
    while edges[-1] < n:
        edges.append(min(n, edges[-1] * 2))
    return list(zip(edges[:-1], edges[1:]))


def units(name, per_stratum=96, threads=None, exact_below=5000, seed=1, pll_below=1_000_000,
          eta=0):
    threads = threads or os.cpu_count()
    g, rank = W.load(name)
    method = "plant_clt" if eta else "plant"
    n = g.n
    order = np.empty(n, np.uint32)
    order[n - 1 - rank.astype(np.int64)] = np.arange(n, dtype=np.uint32)
    t0 = time.time()
    T_exact = n < pll_below and not eta
    T = O.build_labels(g, rank, "pll").total if T_exact else None
    t_pll = time.time() - t0
    rng = np.random.default_rng(seed)
    S = A = Te = 0.0
    varS = varA = varT = 0.0
    sampled = 0
    for lo, hi in strata(n):
        size = hi - lo
        if n <= exact_below or lo == 0 or size <= per_stratum:
            pos = np.arange(lo, hi)
        else:
            pos = np.sort(rng.choice(np.arange(lo, hi), per_stratum, replace=False))
        _, st = O.build_labels(g, rank, method, roots=order[pos], threads=threads, with_stats=True,
                               eta=eta or 16)
        s, a = st[:, 0].astype(np.float64), st[:, 1].astype(np.float64)
        t = st[:, 2].astype(np.float64)
        k = len(pos)
        sampled += k
        S += s.mean() * size
        A += a.mean() * size
        Te += t.mean() * size
        if k < size and k > 1:
            f = (1 - k / size) * size * size / k
            varS += f * s.var(ddof=1)
            varA += f * a.var(ddof=1)
            varT += f * t.var(ddof=1)
    out = {
        "n": int(n), "arcs": int(g.num_arcs), "T": int(T) if T_exact else int(round(Te)),
        "T_exact": bool(T_exact or sampled == n),
        "S": float(S), "A": float(A), "S_stderr": float(varS ** 0.5), "A_stderr": float(varA ** 0.5),
        "roots_sampled": int(sampled), "exact": bool(sampled == n),
        "method": ("T: sequential Algorithm 1; " if T_exact else "T, ") +
                  "S, A: Algorithm 3 with early termination" +
                  (f", pruned by the Common Label Table of the {eta} most important hubs" if eta else "") +
                  ", stratified by rank position (all of the top 64, then doubling strata)",
        "pll_seconds": round(t_pll, 1),
    }
    if not T_exact:
        out["T_stderr"] = float(varT ** 0.5)
    return out


def pll_units(name):
    g, rank = W.load(name)
    L, st = O.build_labels(g, rank, "pll", with_stats=True)
    return {"n": int(g.n), "arcs": int(g.num_arcs), "T": int(L.total), "T_exact": True,
            "S": float(st[:, 0].sum()), "A": float(st[:, 1].sum()), "Q": float(st[:, 3].sum()),
            "S_stderr": 0.0, "A_stderr": 0.0,
            "roots_sampled": int(g.n), "exact": True,
            "method": "sequential Algorithm 1 over all roots (pruned Dijkstra with rank and "
                      "distance queries over all higher-ranked labels)"}


def main(names):
    data = {}
    if os.path.exists(OUT):
        data = json.load(open(OUT))
    for name in names:
        t = time.time()
        if name.endswith("/pll"):
            data[name] = pll_units(name[:-4])
        else:
            base, _, clt = name.partition("/clt")
            data[name] = units(base, eta=int(clt) if clt else 0)
        data[name]["seconds"] = round(time.time() - t, 1)
        print(name, json.dumps(data[name]), flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["ba2k", "rmat18", "grid512"])
