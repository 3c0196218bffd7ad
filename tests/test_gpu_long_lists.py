"""Label lists longer than one shared-memory sort (more than 16,384 labels).

The sort step of Algorithm 2 puts each vertex's labels in hub-rank order
whatever their number. In W.double_star(20000) the lowest-ranked vertex holds
20,002 labels, while the whole labeling has about 60,000, so the long-list
path (chunks sorted in shared memory, then merged) is exercised at a size the
oracle builds in seconds. The GPU labels must equal the oracle's and the
closed form bit for bit.
"""
import os

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
from test_oracle import double_star_closed_form  # noqa: E402


@pytest.fixture(scope="module")
def star():
    chl.build()
    g, rank = W.double_star(20000, seed=11)
    ref = O.build_labels(g, rank, "plant", threads=os.cpu_count() or 1)
    return g, rank, ref


@pytest.mark.parametrize("opts", [dict(), dict(flags=chl.CHL_FLAG_NO_HYBRID),
                                  dict(threads_per_tree=256, label_capacity=1000)])
def test_long_list_bit_exact(star, opts):
    g, rank, ref = star
    L = chl.build_labels(DG(g), dev(rank), **opts)
    off, hub, dist = L.to_numpy()
    assert int(off[1] - off[0]) == g.n  # the long list: every leaf, t and c
    assert_same(ref, off, hub, dist)
    c_off, c_hub, c_dist = double_star_closed_form(g, rank)
    assert np.array_equal(off, c_off) and np.array_equal(hub, c_hub) and np.array_equal(dist, c_dist)
    pairs = W.uniform_pairs(g.n, 20000, seed=4)
    pairs[:100, 0] = 0  # many pairs on the long list
    got = L.query(dev(pairs)).cpu().numpy().view(np.uint32)
    assert np.array_equal(got, O.query(ref, rank, pairs))
    L.free()
