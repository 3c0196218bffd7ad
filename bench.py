"""Benchmark of the canonical hub labeling hot path on one GB300.

One step = one whole build of the workload (every tree in hybrid phases, label
emission, per-vertex sort: chl_build) followed by one batch of PPSD queries
(chl_query), inputs resident in device memory. The headline workload is the
batched scale-free build: R-MAT scale 18 (edge factor 16, a=.57, b=c=.19),
largest component, weights U{1..255}, degree rank, 1,000,000 uniform query
pairs. The build is the hybrid: PLaNT trees (Algorithm 3) in the first phase,
then phases whose trees also prune with every label of the earlier phases.

Prints one JSON line (rank 0). Besides the device-timed value it reports:
  e2e           the same step through the C ABI with host buffers (graph and
                rank copied in, labels and answers copied out)
  roofline      the tree kernel's algorithmic bytes / its device time against
                the measured HBM copy bandwidth
  plain         the one-root-per-launch build (mode 1) of the same phases
  cpu_baseline  the CPU oracle running the algorithm the GPU runs (the phased
                method on all host cores, or Algorithm 3 with the Common Label
                Table for builds that never switch), with the same query batch
  no_hybrid     the single-phase batched PLaNT build (every tree Algorithm 3,
                pruned by the 16-hub table only) and its own roofline
  queries       throughput of the batch, and latency of single-query launches
  configs       the same records for the other workloads: Barabasi-Albert
                n=2,000 with 100,000 queries, the 512x512 road-like grid and
                R-MAT scale 21 (with its total label bytes)
  serving       the continuous-batching server under open-loop Poisson load
  clocks        SM clocks and throttle reasons sampled during the timed steps

--impl reference times the CPU oracle arm alone (the same phased build and
query batch on the host cores), on the same workload, metric and unit.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the serving leg runs query batches and builds on separate streams: give each
# stream its own hardware queue (read at context creation), so that a query
# batch is never queued behind a persistent tree kernel of another stream
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

WORKLOAD_TEXT = {
    "rmat18": "R-MAT scale 18, edge factor 16, a=0.57 b=c=0.19, symmetrised, dedup, LCC; "
              "w~U{1..255}; degree rank; all roots claimed in rank order by one persistent "
              "launch per phase",
    "grid512": "512x512 grid, 10% edges deleted, LCC; w=round(1000*U[0.5,1.5)); "
               "rank by paths through v in 256 sampled shortest-path trees",
    "ba2k": "Barabasi-Albert n=2000 m=3; w~U{1..100}; degree rank",
    "rmat21": "R-MAT scale 21, edge factor 16, a=0.57 b=c=0.19, LCC; w~U{1..1000}; degree rank",
}
QUERIES = {"ba2k": 100_000}  # per-step query batch of each workload (default: --queries)

# DRAM read + write bytes of plant_trees_kernel over one whole build (the sum
# of dram__bytes_read.sum + dram__bytes_write.sum over its launches, one ncu
# capture of the current kernel source), keyed by workload, threads per tree,
# bucket width, whether the build ran label-pruned phases, the big-tree
# bucket width setting and the Common Label Table's size; other builds report
# no traffic
TREE_DRAM_BYTES_PER_BUILD = {
    # captured with overlap_phases=-1 (ncu serialises the second stream)
    ("rmat18", 1024, 1, True, 0, 0): 31.955e9 + 8.734e9,
    ("rmat18", 1024, 1, True, 0, 4): 29.428e9 + 8.107e9,
    ("rmat18", 1024, 2, True, 0, 4): 29.785e9 + 8.236e9,
}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def work_units(name):
    p = os.path.join(ROOT, "oracle", "work_units.json")
    if os.path.exists(p):
        return json.load(open(p)).get(name)
    return None


def strata(n):
    e = [0, 64]
    while e[-1] < n:
        e.append(min(n, e[-1] * 2))
    return list(zip(e[:-1], e[1:]))


def metric_name(name):
    return (f"CHL build labels/s (hybrid: batched PLaNT, then label-pruned phases; {name}) "
            f"+ PPSD query batch")


class Clocks:
    """nvidia-smi sampling in the background during the timed region."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                pass
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle arm
def phase_ends(n, first, last=None):
    """The oracle's phase schedule: one tree per host thread first, then phases
    of doubling size; ends at `last` (default n)."""
    last = n if last is None else last
    ends, e = [], max(1, first)
    while e < last:
        ends.append(e)
        e *= 2
    ends.append(last)
    return ends


def cpu_step(g, rank, pairs, threads, budget_s, hybrid=True):
    """One step of the CPU oracle arm: the build the GPU runs, then the query
    batch, on `threads` host threads. Returns a dict with labels, seconds and
    the sample it covers.

    - hybrid builds: the oracle's phased method (Algorithm 3 trees, each phase
      also pruned by every label of the earlier phases), the whole build when
      the graph is small enough for the budget; otherwise its first phase, one
      complete tree per thread (the top roots, the build's largest trees).
    - builds that never switch (grids): Algorithm 3 with the 16-hub Common
      Label Table (the algorithm the GPU runs there) on a stratified root
      sample, each stratum scaled by its size.
    The queries run the oracle's merge over all of `pairs`."""
    import oracle as O
    n = g.n
    out = {"threads": threads}
    t0 = time.perf_counter()
    if hybrid:
        # core-seconds of the whole phased build, about 1.5e-10 * n * arcs
        # (rmat18: 180 core-seconds measured)
        full = 1.5e-10 * n * float(g.num_arcs) / threads < budget_s
        R = n if full else threads
        L = O.build_labels_phased(g, rank, phase_ends(n, threads, R), threads=threads)
        dt = time.perf_counter() - t0
        out.update(labels=int(L.total), build_s=dt, full=bool(full),
                   sample=(f"phased method, whole build ({len(phase_ends(n, threads))} phases, "
                           f"first {threads} roots then doubling)" if full else
                           f"phased method, first phase only: the top {R} roots, one complete "
                           f"tree per host thread (the whole build does not fit the budget)"))
        Lq = L if full else None
    else:
        est, timed, spent, _ = plant_clt_estimate(g, rank, budget_s, threads)
        out.update(labels=None, build_s=est, full=False, spent_s=spent,
                   sample=f"Algorithm 3 with the 16-hub Common Label Table on {timed} roots "
                          f"stratified by rank position ({spent:.1f} s), each stratum scaled by "
                          f"its size to the whole build")
        Lq = None
    if pairs is not None and Lq is not None:
        # the query merge over the labeling this step built (a sampled build
        # has no whole labeling to query)
        t1 = time.perf_counter()
        O.query(Lq, rank, pairs, threads=threads)
        out["query_s"] = time.perf_counter() - t1
        out["queries"] = int(len(pairs))
    return out


def plant_clt_estimate(g, rank, budget_s, threads, eta=16):
    """Algorithm 3 pruned by the Common Label Table of the eta most important
    hubs over a stratified root sample; (estimated full build seconds, roots
    timed, seconds spent, threads). The table's trees are timed once; every
    sample call rebuilds them, so that time is taken off each call."""
    import oracle as O
    n = g.n
    eta = min(eta, n)
    order = np.empty(n, np.uint32)
    order[n - 1 - rank.astype(np.int64)] = np.arange(n, dtype=np.uint32)
    rng = np.random.default_rng(7)
    t = time.perf_counter()
    O.build_labels(g, rank, "plant_clt", roots=order[:eta], threads=threads, eta=eta)
    t_table = time.perf_counter() - t
    est, timed, spent = t_table, 0, t_table
    per = max(8 * threads, 64)
    for lo, hi in strata(n):
        k = min(per, hi - lo)
        pos = np.sort(rng.choice(np.arange(lo, hi), k, replace=False))
        t = time.perf_counter()
        O.build_labels(g, rank, "plant_clt", roots=order[pos], threads=threads, eta=eta)
        dt = time.perf_counter() - t
        spent += dt
        timed += k
        dt = max(dt - t_table, 0.0)
        est += dt / k * (hi - lo)
        if spent > budget_s:
            for lo2, hi2 in strata(n):  # later strata: this stratum's per-root time
                if lo2 >= hi:
                    est += dt / k * (hi2 - lo2)
            break
    return est, timed, spent, threads


def oracle_T(name, fallback):
    """Exact label count of a workload from the oracle's committed work units."""
    return (work_units(f"{name}/pll") or {}).get("T") or fallback


def cpu_record(step, T_full):
    """cpu_baseline of a step: labels/s of build + queries, on what was timed
    (T_full: the whole labeling's size, for a build estimated from a sample)."""
    q = step.get("query_s", 0.0)
    if step["full"]:
        value, labels = step["labels"] / (step["build_s"] + q), step["labels"]
    elif step["labels"] is not None:
        value, labels = step["labels"] / step["build_s"], step["labels"]
    else:
        value, labels = T_full / (step["build_s"] + q), T_full
    rec = {"value": value, "unit": "labels/s", "cores": step["threads"], "kind": "oracle",
           "sample": step["sample"] + (f"; plus the oracle's query merge over the same "
                                       f"{step['queries']:,} pairs ({q:.2f} s)" if "queries" in step
                                       else "; no queries (the labeling is not built whole)"),
           "build_s": step["build_s"], "query_s": step.get("query_s"), "labels": labels}
    return rec


def run_reference(args, g, rank, name):
    import workloads as W
    threads = os.cpu_count() or 1
    pairs = W.uniform_pairs(g.n, QUERIES.get(name, args.queries), seed=2)
    hybrid = name != "grid512"
    # warm-up steps: the first phase only (untimed; loads the oracle and the pages)
    for _ in range(args.warmup):
        import oracle as O
        O.build_labels_phased(g, rank, phase_ends(g.n, threads, min(g.n, threads)), threads=threads)
    times, step = [], None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step = cpu_step(g, rank, pairs, threads, args.cpu_budget, hybrid=hybrid)
        times.append(time.perf_counter() - t0)
    rec = cpu_record(step, oracle_T(name, step["labels"]))
    v = rec["value"]
    line = {
        "impl": "reference", "metric": metric_name(name), "value": v, "unit": "labels/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": float(np.max(times)) * 1000.0, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": name, "description": WORKLOAD_TEXT.get(name, name), "n": g.n,
                   "arcs": g.num_arcs, "queries_per_step": int(len(pairs))},
        "cpu_baseline": rec,
        "same_config": bool(step["full"] and "queries" in step),
        "e2e": {"value": v, "unit": "labels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU legs
def roofline(name, stats, tree_ms, opts, peak, peak_kind):
    """Tree-kernel roofline: algorithmic bytes from the oracle's work units
    (28 B per settled vertex, 16 B per arc, 12 B per label, and 8 B per label
    entry read by distance queries), divided by the tree kernel's device time.
    A label-pruned (hybrid) build is credited with sequential Algorithm 1's
    work (its floor); a build that never prunes by labels with Algorithm 3
    pruned by the Common Label Table."""
    eta = opts.get("common_hubs", 0)
    eta = 16 if eta == 0 else eta
    hybrid = stats.get("label_table_phases", 0) > 0
    wu_plain = work_units(name)
    wu = work_units(f"{name}/pll") if hybrid else (work_units(f"{name}/clt{eta}") if eta > 0
                                                     else wu_plain)
    if not wu:
        return None
    T_units = wu["T"] if wu.get("T_exact") else (wu_plain or wu)["T"]
    algo = 28.0 * wu["S"] + 16.0 * wu["A"] + 12.0 * T_units
    if hybrid:
        algo += 8.0 * wu.get("Q", 0.0)
    ach = algo / (tree_ms / 1000.0) / 1e9
    key = (name, opts.get("threads_per_tree", 0), opts.get("bucket_delta", 0), bool(hybrid),
           opts.get("big_tree_bucket_delta", 0), opts.get("common_hubs", 0))
    traffic = TREE_DRAM_BYTES_PER_BUILD.get(key)
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": traffic,
            "traffic_note": ("DRAM read + write bytes of the tree kernel over one whole build "
                             "(all its launches), from one ncu capture of the same build and "
                             "launch parameters; per build, like achieved" if traffic else
                             "null: no ncu capture of this workload and these launch parameters "
                             "with the current kernel"),
            "peak_kind": peak_kind, "kernel": "plant_trees_kernel", "algorithmic_bytes": algo,
            "units": ("oracle sequential Algorithm 1 (the label-pruned build's floor)" if hybrid
                      else f"oracle Algorithm 3 pruned by the Common Label Table of {eta} hubs")}


def query_roofline(L, pairs_h, batch_ms, peak):
    """Algorithmic bytes of a query batch: pair 8 + answer 4 + both lists
    scanned to the end (hub position 4 + distance 4 per entry)."""
    off_h = L.to_numpy()[0].astype(np.int64)
    lens = off_h[1:] - off_h[:-1]
    qbytes = 12.0 * len(pairs_h) + 8.0 * float(lens[pairs_h[:, 0]].sum() + lens[pairs_h[:, 1]].sum())
    ach = qbytes / (batch_ms / 1000.0) / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "kernel": "query_kernel", "algorithmic_bytes": qbytes}


class Ctx:
    """Device, stream and event helpers shared by the legs."""

    def __init__(self, torch, chl, local):
        self.torch, self.chl = torch, chl
        self.dev = torch.device("cuda", local)
        self.stream = torch.cuda.current_stream(self.dev)
        self.ev0 = torch.cuda.Event(enable_timing=True)
        self.ev1 = torch.cuda.Event(enable_timing=True)
        self.flush = torch.empty(256 << 20, dtype=torch.uint8, device=self.dev)  # > L2 (129 MB)

    def t(self, a):
        a = np.ascontiguousarray(a)
        return self.torch.from_numpy(a.view(np.int64 if a.dtype == np.uint64 else np.int32)).to(self.dev)

    def sync(self):
        self.torch.cuda.synchronize(self.dev)

    def device_graph(self, g):
        t = self.t

        class DG:
            n = g.n
            row_ptr = t(g.row_ptr)
            col = t(g.col)
            w = t(g.w)
        return DG

    def timed(self, fn):
        self.ev0.record(self.stream)
        r = fn()
        self.ev1.record(self.stream)
        self.sync()
        return r, self.ev0.elapsed_time(self.ev1)


def e2e_leg(cx, g, rank, pairs_h, opts, steps):
    """The step through the C ABI with host buffers: graph and rank copied in,
    labels and answers copied out, all inside the timed region."""
    chl = cx.chl
    pin = lambda a: cx.torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()

    class HG:
        n = g.n
        row_ptr = pin(g.row_ptr)
        col = pin(g.col)
        w = pin(g.w)

    rank_h, pairs_p = pin(rank), pin(pairs_h)
    out_h = pin(np.empty(len(pairs_h), np.uint32))
    times, T = [], 0
    for _ in range(steps):
        cx.sync()
        t0 = time.perf_counter()
        Lh = chl.build_labels(HG, rank_h, **opts)
        off, hub, dist_ = Lh.to_numpy()
        Lh.query(pairs_p, out=out_h)
        cx.sync()
        times.append(time.perf_counter() - t0)
        T = Lh.total
        Lh.free()
    h2d = g.row_ptr.nbytes + g.col.nbytes + g.w.nbytes + rank.nbytes + pairs_h.nbytes
    d2h = off.nbytes + hub.nbytes + dist_.nbytes + out_h.nbytes
    return {"value": T / max(times), "unit": "labels/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": max(times) * 1000.0}


def plain_leg(cx, g, DG, R, opts, stats, tree_ms, max_roots=300_000):
    """The one-root-per-launch form (mode 1) on the same graph: for a hybrid
    build the whole build with the same phases and pruning; otherwise 8
    consecutive roots per rank-position stratum, scaled by stratum size."""
    chl = cx.chl
    if stats.get("label_table_phases", 0) > 0:
        if g.n > max_roots:
            return {"skipped": f"{g.n:,} sequential single-tree launches; not timed"}
        cx.sync()
        Lp = chl.build_labels(DG, R, mode=1, **{k: v for k, v in opts.items() if k != "slots"})
        cx.sync()
        s = Lp.stats()
        Lp.free()
        return {"tree_s": s["tree_ms"] / 1000.0, "roots_timed": g.n, "batched_tree_s": tree_ms / 1000.0,
                "speedup_batched_vs_plain": s["tree_ms"] / tree_ms, "phases": s["phases"],
                "label_table_phases": s["label_table_phases"],
                "how": "mode=1 (one CTA per launch, one launch per root) over every root, with "
                       "the same hybrid phases and pruning"}
    n = g.n
    est, timed, table = 0.0, 0, 0.0
    rng = np.random.default_rng(3)
    for lo, hi in strata(n):
        k = min(8, hi - lo)
        b = int(rng.integers(lo, hi - k + 1))
        cx.sync()
        Lp = chl.build_labels(DG, R, mode=1, root_begin=b, root_end=b + k,
                              common_hubs=opts.get("common_hubs", 0))
        cx.sync()
        s = Lp.stats()
        Lp.free()
        table = max(table, s["table_ms"] / 1000.0)  # a plain build makes its table once
        est += (s["tree_ms"] - s["table_ms"]) / 1000.0 / k * (hi - lo)
        timed += k
    est += table
    return {"est_tree_s": est, "roots_timed": timed, "batched_tree_s": tree_ms / 1000.0,
            "speedup_batched_vs_plain": est / (tree_ms / 1000.0),
            "how": "mode=1 (one CTA per launch, one launch per root) on 8 consecutive roots per "
                   "rank-position stratum, scaled by stratum size"}


def config_leg(cx, name, args, peak, peak_kind, g=None, rank=None, keep=False):
    """One workload's record: tuned build + query batch timed on the device
    (inputs resident), roofline, plain form, e2e, CPU baseline."""
    import workloads as W
    chl = cx.chl
    t_load = time.perf_counter()
    if g is None:
        g, rank = W.load(name)
    t_load = time.perf_counter() - t_load
    DG = cx.device_graph(g)
    R = cx.t(rank)
    nq = QUERIES.get(name, args.queries)
    pairs_h = W.uniform_pairs(g.n, nq, seed=2)
    P = cx.t(pairs_h)
    out = cx.torch.empty(nq, dtype=cx.torch.int32, device=cx.dev)
    t0 = time.perf_counter()
    opts, rep = chl.tune(DG, R)
    t_tune = time.perf_counter() - t0
    def step():
        L = chl.build_labels(DG, R, **opts)
        L.query(P, out=out)
        return L

    for _ in range(2):
        step().free()
    steps, tree, build, qms = [], [], [], []
    for _ in range(args.config_steps):
        cx.flush.zero_()
        cx.sync()
        L, ms = cx.timed(step)
        steps.append(ms)
        st = L.stats()
        tree.append(st["tree_ms"])
        build.append(st["build_ms"])
        stats, T, nbytes = st, L.total, L.nbytes
        L.free()
    L = chl.build_labels(DG, R, **opts)
    for _ in range(3):
        _, ms = cx.timed(lambda: L.query(P, out=out))
        qms.append(ms)
    rec = {"workload": name, "description": WORKLOAD_TEXT.get(name, name), "n": g.n,
           "arcs": g.num_arcs, "value": T / (max(steps) / 1000.0), "unit": "labels/s",
           "ms_per_step": max(steps), "steps": args.config_steps, "queries_per_step": nq,
           "build_ms": float(np.mean(build)), "tree_kernel_ms": float(np.mean(tree)),
           "labels": int(T), "label_bytes": int(nbytes), "als": T / g.n,
           "trees_per_s": g.n / (float(np.mean(build)) / 1000.0), "tuned": opts,
           "tune_s": t_tune, "load_s": t_load,
           "explored": {k: stats[k] for k in ("expanded", "arcs", "pruned", "phases",
                                                "label_table_phases")},
           "queries": {"batch": nq, "queries_per_s": nq / (min(qms) / 1000.0), "batch_ms": min(qms)},
           "query_roofline": query_roofline(L, pairs_h, min(qms), peak),
           "roofline": roofline(name, stats, float(np.mean(tree)), opts, peak, peak_kind)}
    if not args.no_extras:
        rec["plain"] = plain_leg(cx, g, DG, R, opts, stats, float(np.mean(tree)))
        rec["e2e"] = e2e_leg(cx, g, rank, pairs_h, opts, 1)
        cpu = cpu_step(g, rank, pairs_h, os.cpu_count() or 1, args.cpu_budget,
                       hybrid=stats.get("label_table_phases", 0) > 0)
        rec["cpu_baseline"] = cpu_record(cpu, oracle_T(name, T))
    if keep:
        return rec, (g, L)
    L.free()
    return rec, None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat18")
    ap.add_argument("--queries", type=int, default=1_000_000)
    ap.add_argument("--cpu-budget", type=float, default=30.0,
                    help="seconds of host work a CPU baseline may take")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip plain/cpu/e2e/no-hybrid/serving legs")
    ap.add_argument("--configs", default="ba2k,grid512,rmat21",
                    help="other workloads measured after the main one ('none' for none)")
    ap.add_argument("--config-steps", type=int, default=3)
    ap.add_argument("--serve-sets", default="main,rmat21",
                    help="label sets resident in the serving run: 'main' (the bench build) "
                         "and/or workload names, comma separated (e.g. main,rmat21)")
    ap.add_argument("--serve-duration", type=float, default=0.1,
                    help="seconds of Poisson arrivals per offered rate")
    ap.add_argument("--serve-builds", type=int, default=8)
    ap.add_argument("--serve-only", action="store_true",
                    help="build the serving sets and run only the serving leg")
    ap.add_argument("--case", default=None,
                    help="profiling case: one build of the roots at rank positions [b, b+count), "
                         "given as b:count; prints its counters and exits")
    ap.add_argument("--opts", default=None,
                    help="build options k=v,... (e.g. threads_per_tree=256,bucket_delta=1); "
                         "skips the tuner")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank_id = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    import workloads as W
    name = args.workload
    g, rank = W.load(name)

    if args.impl == "reference":
        if rank_id == 0:
            run_reference(args, g, rank, name)
        return

    import torch
    import paper_1907_00140_gb300 as chl
    chl.build()
    torch.cuda.set_device(local)
    cx = Ctx(torch, chl, local)
    dev = cx.dev
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    DG = cx.device_graph(g)
    R = cx.t(rank)
    nq = QUERIES.get(name, args.queries)
    pairs_h = W.uniform_pairs(g.n, nq, seed=2)
    P = cx.t(pairs_h)
    out = torch.empty(nq, dtype=torch.int32, device=dev)
    stream = cx.stream

    # search parameters measured once for this graph (chl_tune), outside the timed region
    if args.opts:
        opts = {k: (float(v) if any(c in v for c in ".eE") else int(v))
                for k, v in (kv.split("=") for kv in args.opts.split(","))}
        tune_rep = {"trials": 0, "sample_roots": 0}
    else:
        opts, tune_rep = chl.tune(DG, R)
    if args.serve_only:
        L = chl.build_labels(DG, R, **opts)
        res = {"metric": "serving", "config": {"workload": name, "tuned": opts},
               "serving": serving_leg(args, chl, g, L, {}, DG, R, P)}
        L.free()
        print(json.dumps(res), flush=True)
        return
    if args.case:
        b, c = (int(x) for x in args.case.split(":"))
        cx.sync()
        L = chl.build_labels(DG, R, root_begin=b, root_end=min(g.n, b + c), **opts)
        st = L.stats()
        L.free()
        print(json.dumps({"case": name, "roots": [b, min(g.n, b + c)], "opts": opts,
                          **{k: st[k] for k in ("tree_ms", "build_ms", "expanded", "arcs",
                                                "labels", "trees", "phases",
                                                "label_table_phases")}}), flush=True)
        return

    def step():
        L = chl.build_labels(DG, R, **opts)
        L.query(P, out=out)
        return L

    def barrier():
        cx.sync()
        if pg:
            pg.barrier()

    for _ in range(args.warmup):
        step().free()
    barrier()

    clocks = Clocks(local)
    times, tree_ms, build_ms, launches = [], [], [], []
    for _ in range(args.steps):
        cx.flush.zero_()
        barrier()
        cx.ev0.record(stream)
        L = step()
        cx.ev1.record(stream)
        cx.sync()
        times.append(cx.ev0.elapsed_time(cx.ev1))
        st = L.stats()
        tree_ms.append(st["tree_ms"])
        build_ms.append(st["build_ms"])
        launches.append(st["launches"] + 1)
        T = st["labels"]
        stats = st
        L.free()
    barrier()
    clk = clocks.stop()
    ms = float(np.max(times))
    if pg:
        x = torch.tensor([ms], device=dev)
        pg.all_reduce(x, op=pg.ReduceOp.MAX)
        ms = float(x.item())

    if rank_id != 0:
        pg.barrier()
        return

    peak, peak_kind = load_peaks()
    value = world * T / (ms / 1000.0)
    res = {
        "metric": metric_name(name), "value": value, "unit": "labels/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": name, "description": WORKLOAD_TEXT.get(name, name), "n": g.n,
                   "arcs": g.num_arcs, "queries_per_step": nq,
                   "l2": "256 MiB buffer written between timed steps; per-step state > L2",
                   "replicas": world, "tuned": opts,
                   "tune": {"trials": tune_rep["trials"], "sample_roots": tune_rep["sample_roots"]}},
        "build_s": float(np.mean(build_ms)) / 1000.0,
        "tree_kernel_ms": float(np.mean(tree_ms)),
        "labels": int(T), "als": T / g.n,
        "trees_per_s": g.n / (float(np.mean(build_ms)) / 1000.0),
        "explored": {"expanded": stats["expanded"], "arcs": stats["arcs"],
                     "trivial": stats["trivial"], "pruned": stats["pruned"],
                     "phases": stats["phases"], "label_table_phases": stats["label_table_phases"]},
        "gpu_launches": int(max(launches)),
        "clocks": clk,
        "roofline": roofline(name, stats, float(np.mean(tree_ms)), opts, peak, peak_kind),
    }

    # ---- queries: batch throughput and single-query launch latency
    L = chl.build_labels(DG, R, **opts)
    qt = [cx.timed(lambda: L.query(P, out=out))[1] for _ in range(5)]
    one = torch.empty(1, dtype=torch.int32, device=dev)
    lat = []
    for i in range(2000):
        p1 = P[i:i + 1]
        cx.ev0.record(stream)
        L.query(p1, out=one)
        cx.ev1.record(stream)
        cx.ev1.synchronize()
        lat.append(cx.ev0.elapsed_time(cx.ev1) * 1000.0)
    res["query_roofline"] = query_roofline(L, pairs_h, min(qt), peak)
    res["queries"] = {"batch": nq, "queries_per_s": nq / (min(qt) / 1000.0),
                      "batch_ms": min(qt), "single_launch_p50_us": float(np.percentile(lat, 50)),
                      "single_launch_p99_us": float(np.percentile(lat, 99)),
                      "single_launch_p999_us": float(np.percentile(lat, 99.9))}

    kept = {}
    if not args.no_extras:
        res["plain"] = plain_leg(cx, g, DG, R, opts, stats, float(np.mean(tree_ms)))
        res["e2e"] = e2e_leg(cx, g, rank, pairs_h, opts, args.steps)
        cpu = cpu_step(g, rank, pairs_h, os.cpu_count() or 1, args.cpu_budget,
                       hybrid=stats.get("label_table_phases", 0) > 0)
        res["cpu_baseline"] = cpu_record(cpu, oracle_T(name, T))
        # ---- the single-phase batched PLaNT build (no label-pruned phases)
        flags = opts.get("flags", 0) | chl.CHL_FLAG_NO_HYBRID
        # the paper's 16-hub table (a tuned smaller one is for the label-pruned phases)
        o1 = dict({k: v for k, v in opts.items() if k != "common_hubs"}, flags=flags)
        chl.build_labels(DG, R, **o1).free()
        Ln, msn = cx.timed(lambda: chl.build_labels(DG, R, **o1))
        sn = Ln.stats()
        Ln.free()
        res["no_hybrid"] = {"build_ms": msn, "tree_kernel_ms": sn["tree_ms"], "labels": sn["labels"],
                            "value": sn["labels"] / (msn / 1000.0), "unit": "labels/s",
                            "expanded": sn["expanded"], "arcs": sn["arcs"], "pruned": sn["pruned"],
                            "roofline": roofline(name, sn, sn["tree_ms"], o1, peak, peak_kind),
                            "how": "CHL_FLAG_NO_HYBRID: every tree in one persistent launch, "
                                   "Algorithm 3 pruned by the 16-hub Common Label Table only"}
    # ---- the other workloads
    configs = [c for c in args.configs.split(",") if c and c != "none" and c != name]
    if configs:
        res["configs"] = {}
        for c in configs:
            t0 = time.perf_counter()
            rec, keep = config_leg(cx, c, args, peak, peak_kind, keep=c in args.serve_sets.split(","))
            rec["leg_s"] = time.perf_counter() - t0
            res["configs"][c] = rec
            if keep:
                kept[c] = keep
    if not args.no_extras and rank_id == 0:
        res["serving"] = serving_leg(args, chl, g, L, kept, DG, R, P)
    L.free()
    for _, Lk in kept.values():
        Lk.free()
    print(json.dumps(res), flush=True)
    if pg:
        pg.barrier()


# ---------------------------------------------------------------- serving
def make_stream(sets, lam, duration, seed):
    """Open-loop Poisson query stream at lam queries/s over `duration` seconds:
    requests of geometric size (mean max(1, lam / 1e6) pairs, so at most about
    a million requests per second), each on a label set chosen uniformly, its
    pairs half uniform, half with both endpoints drawn by degree."""
    import workloads as W
    rng = np.random.default_rng(seed)
    mean = max(1.0, lam / 1e6)
    nreq = max(1, int(round(duration * lam / mean)))
    arr = np.cumsum(rng.exponential(mean / lam, nreq))
    sizes = rng.geometric(1.0 / mean, nreq) if mean > 1 else np.ones(nreq, np.int64)
    set_of = rng.integers(0, len(sets), nreq).astype(np.uint32)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    pairs = np.empty((int(off[-1]), 2), np.uint32)
    for k, (g, _L) in enumerate(sets):
        sel = np.repeat(set_of == k, sizes)
        q = int(sel.sum())
        if not q:
            continue
        half = q // 2
        pk = np.concatenate([W.uniform_pairs(g.n, half, seed + 17 * k),
                             W.degree_pairs(g, q - half, seed + 17 * k + 1)])
        pairs[sel] = pk[rng.permutation(q)]
    return arr, set_of, off, pairs


def run_serving(chl, sets, rates, duration, builds, seed=40):
    """Serving loop under open-loop Poisson load: continuous batching vs the
    plain one-launch-per-request server, and a run with the 8 Barabasi-Albert
    build requests arriving during the stream."""
    import threading
    import workloads as W
    out = {"sets": [g.name for g, _ in sets], "rates": []}

    def one(server, lam, dur, sd):
        arr, so, off, pairs = make_stream(sets, lam, dur, sd)
        before = server.stats()
        ans, lat, wall = server.replay(arr, so, off, pairs)
        after = server.stats()
        nb = after["batches"] - before["batches"]
        return {"offered_qps": lam, "queries": int(off[-1]), "requests": len(arr),
                "achieved_qps": float(off[-1]) / max(wall, 1e-9), "wall_s": wall,
                "p50_us": float(np.percentile(lat, 50) * 1e6),
                "p99_us": float(np.percentile(lat, 99) * 1e6),
                "p999_us": float(np.percentile(lat, 99.9) * 1e6),
                "max_us": float(lat.max() * 1e6), "max_at_s": float(arr[int(lat.argmax())]),
                "batches": int(nb), "mean_batch": float(off[-1]) / max(nb, 1)}, (ans, so, off, pairs)

    S = chl.Server(query_slots=3)
    for _, L in sets:
        S.add_set(L)
    one(S, 1e6, 0.02, seed)  # warm-up
    for i, lam in enumerate(rates):
        r, _ = one(S, lam, duration, seed + i)
        out["rates"].append(r)
    # builds arriving during a stream at 10M queries/s
    bgs = [W.serving_ba(i) for i in range(builds)]
    tickets, lat_b = [], []
    lam, dur = 1e7, max(duration, 0.5)

    def submit():
        for i, (g, r) in enumerate(bgs):
            time.sleep(dur / max(builds, 1))
            tickets.append(S.submit_build(g, r))
    th = threading.Thread(target=submit)
    th.start()
    r, _ = one(S, lam, dur, seed + 99)
    th.join()
    for t in tickets:
        Lb, lt = S.wait(t)
        lat_b.append(lt)
        Lb.free()
    r["builds"] = {"count": len(tickets), "graphs_n": [g.n for g, _ in bgs],
                   "latency_s": [round(x, 4) for x in lat_b]}
    out["with_builds"] = r
    out["server"] = S.stats()
    S.close()
    # plain: one launch per request, each waited for before the next
    P = chl.Server(batching=1)
    for _, L in sets:
        P.add_set(L)
    plain = []
    for lam, dur in ((2e4, 0.25), (1e6, 0.02)):
        r, _ = one(P, lam, dur, seed + 7)
        plain.append(r)
    P.close()
    out["plain"] = plain
    return out


def query_modes(chl, g, L, DG, R, sets, duration, pairs_d):
    """The paper's query modes (Sec. 6) on one GPU beside the default merge:
    - partitioned (QFDL-style): the main labels built again as hub partitions
      (disjoint root ranges), each query the minimum over the parts;
    - grouped (QDOL-style): batches counting-sorted by the vertex blocks their
      pairs read, answers put back in arrival order.
    Reported: the bench's query batch through each entry point (device
    buffers, CUDA events), and the server under open-loop load at 1e7 and 1e8
    queries/s with each mode on the main label set."""
    import torch
    n = g.n
    cuts = sorted({min(n, c) for c in (0, 152, 1216, 9728, n)})
    t0 = time.perf_counter()
    parts = [chl.build_labels(DG, R, root_begin=b, root_end=e) for b, e in zip(cuts[:-1], cuts[1:])]
    build_s = time.perf_counter() - t0
    out = {"partition_root_ranges": [[b, e] for b, e in zip(cuts[:-1], cuts[1:])],
           "partition_build_s": build_s}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    o = torch.empty(pairs_d.shape[0], dtype=torch.int32, device=pairs_d.device)

    def batch(fn):
        ms = []
        for _ in range(4):
            ev0.record()
            fn()
            ev1.record()
            torch.cuda.synchronize()
            ms.append(ev0.elapsed_time(ev1))
        best = min(ms[1:])
        return {"batch_ms": best, "queries_per_s": pairs_d.shape[0] / (best / 1000.0)}

    q = pairs_d.shape[0]
    out["batch"] = {"pairs": q,
                    "merge": batch(lambda: L.query(pairs_d, out=o)),
                    "grouped": batch(lambda: L.query(pairs_d, out=o, grouped=True)),
                    "partitioned": batch(lambda: chl.query_partitioned(parts, pairs_d, out=o))}
    main = [(g, L)]
    res = {}
    for mode, make in (("merge", lambda: chl.Server(query_slots=3)),
                       ("grouped", lambda: chl.Server(query_slots=3, query_order=1)),
                       ("partitioned", lambda: chl.Server(query_slots=3))):
        S = make()
        if mode == "partitioned":
            S.add_partitioned_set(parts)
        else:
            S.add_set(L)
        S.replay(*make_stream(main, 1e6, 0.01, 699))  # warm-up
        rows = []
        for i, lam in enumerate((1e7, 1e8)):
            arr, so, off, pairs = make_stream(main, lam, duration, 700 + i)
            ans, lat, wall = S.replay(arr, so, off, pairs)
            rows.append({"offered_qps": lam, "queries": int(off[-1]),
                         "achieved_qps": float(off[-1]) / max(wall, 1e-9),
                         "p50_us": float(np.percentile(lat, 50) * 1e6),
                         "p99_us": float(np.percentile(lat, 99) * 1e6),
                         "p999_us": float(np.percentile(lat, 99.9) * 1e6)})
        S.close()
        res[mode] = rows
    out["serving"] = res
    for x in parts:
        x.free()
    return out


def serving_leg(args, chl, g, L, kept, DG, R, P):
    """Serving run over the bench's labels and other workloads' labels (those
    the config legs kept, else built here)."""
    import workloads as W
    sets, extra, builds_info = [], [], []
    for nm in args.serve_sets.split(","):
        if nm == "main":
            sets.append((g, L))
            continue
        if nm in kept:
            sets.append(kept[nm])
            continue
        g2, r2 = W.load(nm)
        o2, _rep = chl.tune(g2, r2)
        L2 = chl.build_labels(g2, r2, **o2)
        st2 = L2.stats()
        builds_info.append({"workload": nm, "n": g2.n, "tuned": o2, "build_ms": st2["build_ms"],
                            "labels": L2.total, "label_bytes": L2.nbytes})
        extra.append(L2)
        sets.append((g2, L2))
    t0 = time.perf_counter()
    out = run_serving(chl, sets, [1e6, 3e6, 1e7, 3e7, 1e8], args.serve_duration, args.serve_builds)
    out["modes"] = query_modes(chl, g, L, DG, R, sets, args.serve_duration, P)
    out["leg_s"] = time.perf_counter() - t0
    out["label_sets"] = [{"workload": gg.name, "n": gg.n, "labels": LL.total, "bytes": LL.nbytes}
                         for gg, LL in sets]
    out["extra_builds"] = builds_info
    for x in extra:
        x.free()
    return out


if __name__ == "__main__":
    main()
