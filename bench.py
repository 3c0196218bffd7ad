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

WORKLOAD_TEXT = {
    "rmat18": "R-MAT scale 18, edge factor 16, a=0.57 b=c=0.19, symmetrised, dedup, LCC; "
              "w~U{1..255}; degree rank; all roots in one persistent launch",
    "grid512": "512x512 grid, 10% edges deleted, LCC; w=round(1000*U[0.5,1.5)); "
               "rank by paths through v in 256 sampled shortest-path trees",
    "ba2k": "Barabasi-Albert n=2000 m=3; w~U{1..100}; degree rank",
    "rmat21": "R-MAT scale 21, edge factor 16, a=0.57 b=c=0.19, LCC; w~U{1..1000}; degree rank",
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
        opts = {k: int(v) for k, v in (kv.split("=") for kv in args.opts.split(","))}
        tune_rep = {"trials": 0, "sample_roots": 0}
    else:
        opts, tune_rep = chl.tune(DG, R)
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
                     "trivial": stats["trivial"]},
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
    res["queries"] = {"batch": args.queries, "queries_per_s": args.queries / (min(qt) / 1000.0),
                      "batch_ms": min(qt), "single_launch_p50_us": float(np.percentile(lat, 50)),
                      "single_launch_p99_us": float(np.percentile(lat, 99)),
                      "single_launch_p999_us": float(np.percentile(lat, 99.9))}

    # ---- roofline of the tree kernel (algorithmic bytes per SURVEY-style unit counts)
    peak, peak_kind = load_peaks()
    # the build prunes with the Common Label Table of 16 hubs unless told otherwise
    eta = opts.get("common_hubs", 0)
    eta = 16 if eta == 0 else eta
    wu_plain = work_units(name)
    wu = work_units(f"{name}/clt{eta}") if eta > 0 else wu_plain
    if wu and wu_plain:
        algo = 28.0 * wu["S"] + 16.0 * wu["A"] + 12.0 * wu_plain["T"]
        ach = algo / (float(np.mean(tree_ms)) / 1000.0) / 1e9
        res["roofline"] = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                           "frac": ach / peak, "traffic": None, "peak_kind": peak_kind,
                           "kernel": "plant_trees_kernel",
                           "algorithmic_bytes": algo,
                           "units": (f"oracle Algorithm 3 pruned by the Common Label Table of {eta} hubs"
                                     if eta > 0 else "oracle Algorithm 3")}

    if not args.no_extras:
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
    L.free()
    print(json.dumps(res), flush=True)
    if pg:
        pg.barrier()


if __name__ == "__main__":
    main()
