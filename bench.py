"""Benchmark of the canonical hub labeling hot path on one GB300.

One step = one PLaNT build of the whole workload (every tree, label emission,
per-vertex sort: chl_build) followed by one batch of PPSD queries
(chl_query), inputs resident in device memory. The default workload is the
batched scale-free build: R-MAT scale 18 (edge factor 16, a=.57, b=c=.19),
largest component, weights U{1..255}, degree rank, 1,000,000 uniform query
pairs.

Prints one JSON line (rank 0). Besides the device-timed value it reports:
  e2e           the same step through the C ABI with host buffers (graph and
                rank copied in, labels and answers copied out)
  roofline      the tree kernel's algorithmic bytes / its device time against
                the measured HBM copy bandwidth
  plain         the one-root-per-launch build (mode 1), timed on stratified
                root samples and scaled to the whole workload
  cpu_baseline  the CPU oracle (Algorithm 3, all host cores, dynamic root
                claiming) on a bounded stratified root sample, scaled likewise
  queries       throughput of the batch, and latency of single-query launches
  clocks        SM clocks and throttle reasons sampled during the timed steps

--impl reference times the CPU oracle arm alone (the paper's method as the
plain CPU program), on the same workload, metric and unit.
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
              "w~U{1..255}; degree rank; all roots in one persistent launch",
    "grid512": "512x512 grid, 10% edges deleted, LCC; w=round(1000*U[0.5,1.5)); "
               "rank by paths through v in 256 sampled shortest-path trees",
    "ba2k": "Barabasi-Albert n=2000 m=3; w~U{1..100}; degree rank",
    "rmat21": "R-MAT scale 21, edge factor 16, a=0.57 b=c=0.19, LCC; w~U{1..1000}; degree rank",
}


# DRAM read + write bytes of plant_trees_kernel over one whole build (the sum
# of dram__bytes_read.sum + dram__bytes_write.sum over its 11 launches, one ncu
# capture of the current kernel source), keyed by workload and the launch
# parameters it was taken with; other builds report no traffic
TREE_DRAM_BYTES_PER_BUILD = {
    ("rmat18", 1024, 1, 32): 38.295e9 + 11.475e9,
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


def cpu_oracle_estimate(g, rank, T, budget_s=20.0, threads=None, eta=16):
    """Oracle (Algorithm 3 with early termination, pruned by the Common Label
    Table of the eta most important hubs as the GPU build is, dynamic root
    claiming over all host cores) on a stratified root sample; returns
    (estimated full build seconds, roots timed, seconds spent, cores). The
    table's own trees are timed once; every sample call rebuilds them, so
    that time is taken off each call."""
    import oracle as O
    threads = threads or os.cpu_count()
    n = g.n
    eta = min(eta, n)
    method = "plant_clt" if eta > 0 else "plant"
    order = np.empty(n, np.uint32)
    order[n - 1 - rank.astype(np.int64)] = np.arange(n, dtype=np.uint32)
    rng = np.random.default_rng(7)
    t_table = 0.0
    if eta > 0:
        t = time.perf_counter()
        O.build_labels(g, rank, method, roots=order[:eta], threads=threads, eta=eta)
        t_table = time.perf_counter() - t
    est, timed, spent = t_table, 0, t_table
    per = max(8 * threads, 64)
    for lo, hi in strata(n):
        k = min(per, hi - lo)
        pos = np.sort(rng.choice(np.arange(lo, hi), k, replace=False))
        t = time.perf_counter()
        O.build_labels(g, rank, method, roots=order[pos], threads=threads, eta=max(eta, 1))
        dt = time.perf_counter() - t
        spent += dt
        timed += k
        dt = max(dt - t_table, 0.0)
        est += dt / k * (hi - lo)
        if spent > budget_s:
            # remaining strata: extrapolate from this one's per-root time (smaller trees)
            for lo2, hi2 in strata(n):
                if lo2 >= hi:
                    est += dt / k * (hi2 - lo2)
            break
    return est, timed, spent, threads


def run_reference(args, g, rank, name):
    units = work_units(name) or {}
    import oracle as O
    T = units.get("T") or O.build_labels(g, rank, "pll").total
    vals = []
    info = None
    for i in range(args.warmup + args.steps):
        est, timed, spent, cores = cpu_oracle_estimate(g, rank, T, budget_s=args.cpu_budget)
        if i >= args.warmup:
            vals.append(T / est)
            info = (est, timed, spent, cores)
    v = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": metric_name(name), "value": v, "unit": "labels/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": info[2] * 1000.0, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": name, "description": WORKLOAD_TEXT.get(name, name), "n": g.n,
                   "arcs": g.num_arcs},
        "cpu_baseline": {"value": v, "unit": "labels/s", "cores": info[3], "kind": "oracle",
                         "sample": f"Algorithm 3 with the 16-hub Common Label Table: the table's "
                                   f"trees once, then {info[1]} roots stratified by rank position, "
                                   f"each stratum scaled by its size; est. full build {info[0]:.1f} s"},
        "e2e": {"value": v, "unit": "labels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def metric_name(name):
    return f"CHL build labels/s (batched PLaNT, {name}) + PPSD query batch"


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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat18")
    ap.add_argument("--queries", type=int, default=1_000_000)
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-extras", action="store_true", help="skip plain/cpu/e2e legs")
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
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    def t(a):
        a = np.ascontiguousarray(a)
        return torch.from_numpy(a.view(np.int64 if a.dtype == np.uint64 else np.int32)).to(dev)

    class DG:
        n = g.n
        row_ptr = t(g.row_ptr)
        col = t(g.col)
        w = t(g.w)

    R = t(rank)
    pairs_h = W.uniform_pairs(g.n, args.queries, seed=2)
    P = t(pairs_h)
    out = torch.empty(args.queries, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream(dev)

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
               "serving": serving_leg(args, chl, g, L, DG, R)}
        L.free()
        print(json.dumps(res), flush=True)
        return
    if args.case:
        b, c = (int(x) for x in args.case.split(":"))
        torch.cuda.synchronize(dev)
        L = chl.build_labels(DG, R, root_begin=b, root_end=min(g.n, b + c), **opts)
        st = L.stats()
        L.free()
        print(json.dumps({"case": name, "roots": [b, min(g.n, b + c)], "opts": opts,
                          **{k: st[k] for k in ("tree_ms", "build_ms", "expanded", "arcs",
                                                "labels", "trees")}}), flush=True)
        return

    def step():
        L = chl.build_labels(DG, R, **opts)
        L.query(P, out=out)
        return L

    def barrier():
        torch.cuda.synchronize(dev)
        if pg:
            pg.barrier()

    for _ in range(args.warmup):
        L = step()
        L.free()
    barrier()

    clocks = Clocks(local)
    times, tree_ms, build_ms, launches, Ls = [], [], [], [], []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        flush.zero_()
        barrier()
        ev0.record(stream)
        L = step()
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        times.append(ev0.elapsed_time(ev1))
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

    value = world * T / (ms / 1000.0)
    res = {
        "metric": metric_name(name), "value": value, "unit": "labels/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": name, "description": WORKLOAD_TEXT.get(name, name), "n": g.n,
                   "arcs": g.num_arcs, "queries_per_step": args.queries,
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
    }

    # ---- queries: batch throughput and single-query launch latency
    L = chl.build_labels(DG, R, **opts)
    qt = []
    for _ in range(5):
        ev0.record(stream)
        L.query(P, out=out)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        qt.append(ev0.elapsed_time(ev1))
    one = torch.empty(1, dtype=torch.int32, device=dev)
    lat = []
    for i in range(2000):
        p1 = P[i:i + 1]
        ev0.record(stream)
        L.query(p1, out=one)
        ev1.record(stream)
        ev1.synchronize()
        lat.append(ev0.elapsed_time(ev1) * 1000.0)
    # algorithmic bytes of the batch: pair 8 + answer 4 + both lists scanned to the end
    # (hub position 4 + distance 4 per entry), from the label offsets
    off_h = L.to_numpy()[0].astype(np.int64)
    lens = off_h[1:] - off_h[:-1]
    qbytes = 12.0 * args.queries + 8.0 * float(lens[pairs_h[:, 0]].sum() + lens[pairs_h[:, 1]].sum())
    qach = qbytes / (min(qt) / 1000.0) / 1e9
    peak_q, _ = load_peaks()
    res["query_roofline"] = {"bound": "hbm", "achieved": qach, "peak": peak_q, "unit": "GB/s",
                             "frac": qach / peak_q, "kernel": "query_kernel",
                             "algorithmic_bytes": qbytes}
    res["queries"] = {"batch": args.queries, "queries_per_s": args.queries / (min(qt) / 1000.0),
                      "batch_ms": min(qt), "single_launch_p50_us": float(np.percentile(lat, 50)),
                      "single_launch_p99_us": float(np.percentile(lat, 99)),
                      "single_launch_p999_us": float(np.percentile(lat, 99.9))}

    # ---- roofline of the tree kernel (algorithmic bytes from per-unit work counts)
    peak, peak_kind = load_peaks()
    # the build prunes with the Common Label Table of 16 hubs unless told otherwise
    eta = opts.get("common_hubs", 0)
    eta = 16 if eta == 0 else eta
    wu_plain = work_units(name)
    wu = work_units(f"{name}/clt{eta}") if eta > 0 else wu_plain
    hybrid = stats.get("label_table_phases", 0) > 0
    if hybrid:
        # the label-pruned build: credited with sequential Algorithm 1's work,
        # its floor (batched phases see staler tables; that overhead is not credited)
        wu = work_units(f"{name}/pll")
    if wu and wu_plain:
        T_units = wu["T"] if wu.get("T_exact") else wu_plain["T"]
        algo = 28.0 * wu["S"] + 16.0 * wu["A"] + 12.0 * T_units
        if hybrid:
            # plus the label entries (hub, dist: 8 B) its distance queries read
            algo += 8.0 * wu.get("Q", 0.0)
        ach = algo / (float(np.mean(tree_ms)) / 1000.0) / 1e9
        key = (name, opts.get("threads_per_tree", 1024), opts.get("bucket_delta", 0),
               opts.get("window_buckets", 32))
        traffic = TREE_DRAM_BYTES_PER_BUILD.get(key)
        res["roofline"] = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                           "frac": ach / peak,
                           "traffic": traffic,
                           "traffic_note": ("DRAM read + write bytes of the tree kernel over one "
                                            "whole build (all its launches), from one ncu capture "
                                            "of the same build and launch parameters; per build, "
                                            "like achieved" if traffic else
                                            "null: no capture of this workload and these launch "
                                            "parameters with the current kernel"),
                           "peak_kind": peak_kind,
                           "kernel": "plant_trees_kernel",
                           "algorithmic_bytes": algo,
                           "units": ("oracle sequential Algorithm 1 (the label-pruned build's floor)"
                                     if hybrid else
                                     f"oracle Algorithm 3 pruned by the Common Label Table of {eta} hubs"
                                     if eta > 0 else "oracle Algorithm 3")}

    if not args.no_extras and stats.get("label_table_phases", 0) > 0:
        # ---- plain form of the hybrid build: the whole build, one launch per root
        torch.cuda.synchronize(dev)
        Lp = chl.build_labels(DG, R, mode=1, **{k: v for k, v in opts.items() if k != "slots"})
        torch.cuda.synchronize(dev)
        s = Lp.stats()
        Lp.free()
        res["plain"] = {"tree_s": s["tree_ms"] / 1000.0, "roots_timed": g.n,
                        "batched_tree_s": float(np.mean(tree_ms)) / 1000.0,
                        "speedup_batched_vs_plain": s["tree_ms"] / float(np.mean(tree_ms)),
                        "phases": s["phases"], "label_table_phases": s["label_table_phases"],
                        "how": "mode=1 (one CTA per launch, one launch per root) over every root, "
                               "with the same hybrid phases and pruning"}
    elif not args.no_extras:
        # ---- plain one-root-per-launch form on stratified samples
        n = g.n
        est, timed, table = 0.0, 0, 0.0
        rng = np.random.default_rng(3)
        for lo, hi in strata(n):
            k = min(8, hi - lo)
            b = int(rng.integers(lo, hi - k + 1))
            torch.cuda.synchronize(dev)
            Lp = chl.build_labels(DG, R, mode=1, root_begin=b, root_end=b + k,
                                  common_hubs=opts.get("common_hubs", 0))
            torch.cuda.synchronize(dev)
            s = Lp.stats()
            Lp.free()
            # a plain build makes its table once; each sample call rebuilt it
            table = max(table, s["table_ms"] / 1000.0)
            est += (s["tree_ms"] - s["table_ms"]) / 1000.0 / k * (hi - lo)
            timed += k
        est += table
        res["plain"] = {"est_tree_s": est, "roots_timed": timed,
                        "batched_tree_s": float(np.mean(tree_ms)) / 1000.0,
                        "speedup_batched_vs_plain": est / (float(np.mean(tree_ms)) / 1000.0),
                        "how": "mode=1 (one CTA per launch, one launch per root) on 8 "
                               "consecutive roots per rank-position stratum, scaled by stratum size"}
    if not args.no_extras:
        # ---- e2e through the C ABI with host buffers
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()

        class HG:
            n = g.n
            row_ptr = pin(g.row_ptr)
            col = pin(g.col)
            w = pin(g.w)

        rank_h, pairs_p = pin(rank), pin(pairs_h)
        out_h = pin(np.empty(args.queries, np.uint32))
        e2e = []
        for i in range(args.steps):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            Lh = chl.build_labels(HG, rank_h, **opts)
            off, hub, dist_ = Lh.to_numpy()
            Lh.query(pairs_p, out=out_h)
            torch.cuda.synchronize(dev)
            e2e.append(time.perf_counter() - t0)
            Lh.free()
        h2d = g.row_ptr.nbytes + g.col.nbytes + g.w.nbytes + rank.nbytes + pairs_h.nbytes
        d2h = off.nbytes + hub.nbytes + dist_.nbytes + out_h.nbytes
        res["e2e"] = {"value": T / max(e2e), "unit": "labels/s", "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(d2h), "ms_per_step": max(e2e) * 1000.0}
        # ---- CPU oracle baseline (bounded)
        est_c, timed_c, spent_c, cores = cpu_oracle_estimate(g, rank, T, budget_s=args.cpu_budget)
        res["cpu_baseline"] = {"value": T / est_c, "unit": "labels/s", "cores": cores,
                               "kind": "oracle",
                               "sample": f"Algorithm 3 with the 16-hub Common Label Table: "
                                         f"the table's trees once, then {timed_c} roots "
                                         f"stratified by rank position ({spent_c:.1f} s of CPU "
                                         f"work), scaled by stratum size; est. full build "
                                         f"{est_c:.1f} s"}
    if not args.no_extras and rank_id == 0:
        res["serving"] = serving_leg(args, chl, g, L, DG, R)
    L.free()
    print(json.dumps(res), flush=True)
    if pg:
        pg.barrier()


def serving_leg(args, chl, g, L, DG, R):
    """Serving run over the bench's labels and any extra workloads' labels."""
    import workloads as W
    sets, extra, builds_info = [], [], []
    for nm in args.serve_sets.split(","):
        if nm == "main":
            sets.append((g, L))
            continue
        g2, r2 = W.load(nm)
        t0 = time.perf_counter()
        o2, rep2 = chl.tune(g2, r2)
        t1 = time.perf_counter()
        L2 = chl.build_labels(g2, r2, **o2)
        t2 = time.perf_counter()
        st2 = L2.stats()
        builds_info.append({"workload": nm, "n": g2.n, "arcs": g2.num_arcs, "tuned": o2,
                            "tune_s": t1 - t0, "build_wall_s": t2 - t1,
                            "build_ms": st2["build_ms"], "tree_ms": st2["tree_ms"],
                            "table_ms": st2["table_ms"], "sort_ms": st2["sort_ms"],
                            "labels": L2.total, "label_bytes": L2.nbytes,
                            "expanded": st2["expanded"], "arcs_relaxed": st2["arcs"],
                            "pruned": st2["pruned"]})
        extra.append(L2)
        sets.append((g2, L2))
    t0 = time.perf_counter()
    out = run_serving(chl, sets, [1e6, 3e6, 1e7, 3e7, 1e8], args.serve_duration, args.serve_builds)
    out["leg_s"] = time.perf_counter() - t0
    out["label_sets"] = [{"workload": gg.name, "n": gg.n, "labels": LL.total, "bytes": LL.nbytes}
                         for gg, LL in sets]
    out["extra_builds"] = builds_info
    for x in extra:
        x.free()
    return out


if __name__ == "__main__":
    main()
