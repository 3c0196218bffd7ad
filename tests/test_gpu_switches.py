"""GPU parity across the hybrid's switch points (Sec. 5.2): wherever the
first-phase switch (labels per arc, switch_ratio), the Psi switch
(psi_threshold), the small-tree switch (small_tree_expansions) and the
narrow bucket width after big trees (big_tree_bucket_delta) fire, and with or
without the next phase's first trees overlapped with a phase's tail
(overlap_phases), the labels are the canonical ones, bit-exact with the CPU
oracle. Only the amount
of work changes: the label table of earlier phases covers a rank-closed hub
set whenever it is used (Sec. 5.3), and the small-tree launch runs the same
search in smaller blocks. Each build's statistics show which switch fired.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1907_00140_gb300 as chl  # noqa: E402

from test_gpu_parity import DG, dev, assert_same  # noqa: E402

NEVER_SMALL = 1               # no tree averages fewer than one expansion
ALWAYS_SMALL = 0xFFFFFFFF     # every label-pruned phase's trees average fewer


@pytest.fixture(scope="module", autouse=True)
def _built():
    chl.build()
    chl.lib()


def _family(name):
    if name == "ba2k":
        g, rank = W.load("ba2k")
    else:
        g = W.rmat(13, 16, seed=13, whi=255)
        rank = W.degree_rank(g)
    return g, rank, O.build_labels(g, rank, "plant", threads=8)


@pytest.fixture(scope="module", params=["ba2k", "rmat13"])
def family(request):
    g, rank, ref = _family(request.param)
    return request.param, g, rank, ref, DG(g), dev(rank)


# (options, check of the build's statistics)
SWEEP = [
    # first-phase switch on labels per arc: off, never reached, default, always
    (dict(switch_ratio=-1.0), None),
    (dict(switch_ratio=1e-6, psi_threshold=1e9), lambda s: s["label_table_phases"] == 0),
    (dict(), None),
    (dict(switch_ratio=1e6), lambda s: s["label_table_phases"] == s["phases"] - 1),
    # the Psi switch alone (first-phase switch off)
    (dict(switch_ratio=-1.0, psi_threshold=0.5), lambda s: s["label_table_phases"] == s["phases"] - 1),
    (dict(switch_ratio=-1.0, psi_threshold=2.0), None),
    (dict(switch_ratio=-1.0, psi_threshold=1e9), lambda s: s["label_table_phases"] == 0),
    # the small-tree switch: never, default, right after the first label-pruned phase
    (dict(switch_ratio=1e6, small_tree_expansions=NEVER_SMALL), lambda s: s["small_tree_phases"] == 0),
    (dict(switch_ratio=1e6, small_tree_expansions=2048), None),
    (dict(switch_ratio=1e6, small_tree_expansions=ALWAYS_SMALL),
     lambda s: s["small_tree_phases"] == s["label_table_phases"] - 1),
    (dict(switch_ratio=1e6, small_tree_expansions=ALWAYS_SMALL, small_threads_per_tree=64),
     lambda s: s["small_tree_phases"] == s["label_table_phases"] - 1),
    (dict(switch_ratio=1e6, small_tree_expansions=ALWAYS_SMALL, small_threads_per_tree=1024,
          pruned_threads_per_tree=256), lambda s: s["small_tree_phases"] == s["label_table_phases"] - 1),
    # the narrow bucket width after big trees: default, off, set
    (dict(switch_ratio=1e6, big_tree_bucket_delta=-1), None),
    (dict(switch_ratio=1e6, big_tree_bucket_delta=1), None),
    (dict(switch_ratio=1e6, big_tree_bucket_delta=3, pruned_bucket_delta=4096), None),
    # the next phase's first trees in a phase's tail (second stream, older
    # table): off; in every label-pruned phase; with a label buffer so small
    # that their trees overflow it and are built again by their own phase
    (dict(switch_ratio=1e6, overlap_phases=-1), None),
    (dict(switch_ratio=1e6, small_tree_expansions=NEVER_SMALL), lambda s: s["small_tree_phases"] == 0),
    (dict(switch_ratio=1e6, small_tree_expansions=NEVER_SMALL, label_capacity=1000), None),
    (dict(switch_ratio=1e6, small_tree_expansions=NEVER_SMALL, threads_per_tree=256, flags=chl.CHL_FLAG_PARENTS),
     None),
    # smaller Common Label Tables (the tuner's candidates; the label table
    # holds the hubs left out)
    (dict(switch_ratio=1e6, common_hubs=8), None),
    (dict(switch_ratio=1e6, common_hubs=4, small_tree_expansions=NEVER_SMALL), None),
    # both switches with the other block sizes and bucket widths
    (dict(threads_per_tree=256, switch_ratio=1e6, small_tree_expansions=ALWAYS_SMALL,
          pruned_bucket_delta=1), None),
    (dict(threads_per_tree=512, psi_threshold=4.0, small_tree_expansions=512, bucket_delta=2), None),
]


@pytest.mark.parametrize("opts,check", SWEEP, ids=[",".join(f"{k}={v}" for k, v in o.items()) or "default"
                                                    for o, _ in SWEEP])
def test_switch_sweep_is_exact(family, opts, check):
    name, g, rank, ref, G, R = family
    L = chl.build_labels(G, R, **opts)
    st = L.stats()
    assert st["phases"] > 1, st
    assert st["small_tree_phases"] <= st["label_table_phases"], st
    if check is not None:
        assert check(st), (opts, st)
    assert_same(ref, *L.to_numpy())
    L.free()


def test_tuned_switch_points_are_exact(family):
    """chl_tune settles the switch points by whole builds; what it picks
    builds the canonical labels."""
    name, g, rank, ref, G, R = family
    opts, rep = chl.tune(G, R)
    assert rep["trials"] >= 3
    for k in ("switch_ratio", "small_tree_expansions", "big_tree_bucket_delta", "common_hubs"):
        assert k not in opts or opts[k] != 0
    L = chl.build_labels(G, R, **opts)
    assert_same(ref, *L.to_numpy())
    pairs = W.query_pairs(g, 20_000, seed=21)
    got = L.query(dev(pairs)).cpu().numpy().view(np.uint32)
    assert np.array_equal(got, O.query(ref, rank, pairs, threads=8))
    L.free()
