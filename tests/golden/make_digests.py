"""Writes tests/golden/label_digests.json: for each full-size workload the
number of canonical labels and the SHA-256 of the whole labeling (offsets as
little-endian uint64, then hub and distance arrays as little-endian uint32, in
the library's layout: per vertex id, hubs by descending rank). Every value is
computed by the oracle alone, with sequential Algorithm 1 (pruned labeling in
rank order, which reaches the canonical labeling, Sec. 4.1), so a GPU test can
check a full-size build bit for bit without running the oracle.

    python tests/golden/make_digests.py [--inputs-only] [workload ...]
        (default: rmat18 grid512 rmat21; --inputs-only refreshes only the
        input digests and keeps the stored labeling digests)
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

OUT = os.path.join(HERE, "label_digests.json")


def digest(offsets, hub, dist):
    """SHA-256 of a labeling in the library's layout."""
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(offsets, dtype="<u8").tobytes())
    h.update(np.ascontiguousarray(hub, dtype="<u4").tobytes())
    h.update(np.ascontiguousarray(dist, dtype="<u4").tobytes())
    return h.hexdigest()


def input_digest(g, rank):
    """SHA-256 of a workload's inputs (CSR row pointers, columns, weights,
    rank), to tell a generator that differs between machines from a labeling
    that differs."""
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.row_ptr, dtype="<u8").tobytes())
    h.update(np.ascontiguousarray(g.col, dtype="<u4").tobytes())
    h.update(np.ascontiguousarray(g.w, dtype="<u4").tobytes())
    h.update(np.ascontiguousarray(rank, dtype="<u4").tobytes())
    return h.hexdigest()


def main(names, inputs_only=False):
    import oracle as O
    import workloads as W
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        t = time.time()
        g, rank = W.load(name)
        if inputs_only:
            data.setdefault(name, {})["input_sha256"] = input_digest(g, rank)
        else:
            L = O.build_labels(g, rank, "pll")
            data[name] = {"labels": int(L.total), "sha256": digest(L.offsets, L.hub, L.dist),
                          "input_sha256": input_digest(g, rank),
                          "oracle": "sequential Algorithm 1 (build_labels 'pll')",
                          "seconds": round(time.time() - t, 1)}
        print(name, json.dumps(data[name]), flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    args = [a for a in sys.argv[1:] if a != "--inputs-only"]
    main(args or ["rmat18", "grid512", "rmat21"], inputs_only="--inputs-only" in sys.argv)
