"""Host logic of the multi-rank form on CPU (gloo, world size 2): trees are
independent (Sec. 5.2), so ranks that build disjoint root ranges (the ABI's
root_begin/root_end) hold disjoint, hub-partitioned label sets whose union is
the full labeling; the benchmark's step time is the maximum over ranks. The
per-rank labels here come from the oracle (no GPU); the GPU build of a root
range is checked against the oracle's in test_gpu_parity."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def shard(n, world, r):
    """contiguous rank-position range of rank r"""
    return r * n // world, (r + 1) * n // world


def worker(r, world, port, out_path):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle as O
    import workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=r, world_size=world)
    g, rank = W.load("ba2k")
    n = g.n
    order = np.empty(n, np.uint32)
    order[n - 1 - rank.astype(np.int64)] = np.arange(n, dtype=np.uint32)
    rb, re = shard(n, world, r)
    L = O.build_labels(g, rank, "plant", roots=order[rb:re])
    vert = np.repeat(np.arange(n), np.diff(L.offsets.astype(np.int64)))
    trip = torch.from_numpy(np.stack([vert, L.hub, L.dist], 1).astype(np.int64))
    # gather the variable-length label sets of all ranks
    cnt = torch.tensor([len(trip)], dtype=torch.int64)
    cnts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(cnts, cnt)
    m = int(max(c.item() for c in cnts))
    pad = torch.full((m, 3), -1, dtype=torch.int64)
    pad[:len(trip)] = trip
    parts = [torch.zeros((m, 3), dtype=torch.int64) for _ in range(world)]
    dist.all_gather(parts, pad)
    # step time: the maximum over ranks (bench.py's reduction)
    t = torch.tensor([float(r + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if r == 0:
        allp = torch.cat([p[:int(c.item())] for p, c in zip(parts, cnts)]).numpy()
        np.save(out_path, allp)
        assert t.item() == float(world)
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_build_is_hub_partition(tmp_path):
    import oracle as O
    import workloads as W
    world = 2
    out = str(tmp_path / "labels.npy")
    mp.start_processes(worker, args=(world, free_port(), out), nprocs=world, start_method="spawn")
    got = np.load(out)
    g, rank = W.load("ba2k")
    full = O.build_labels(g, rank, "plant")
    vert = np.repeat(np.arange(g.n), np.diff(full.offsets.astype(np.int64)))
    want = np.stack([vert, full.hub, full.dist], 1).astype(np.int64)
    key = lambda a: a[np.lexsort((a[:, 2], a[:, 1], a[:, 0]))]
    assert len(got) == len(want)
    assert np.array_equal(key(got), key(want))
    # the two ranks' hubs are disjoint
    n = g.n
    order = np.empty(n, np.uint32)
    order[n - 1 - rank.astype(np.int64)] = np.arange(n, dtype=np.uint32)
    a, b = set(order[:n // 2].tolist()), set(order[n // 2:].tolist())
    assert not (a & b)
