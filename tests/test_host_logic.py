"""Host-side logic that needs no GPU: the synthetic workloads' promises (seeded,
no repeats, windows slide over live edges), the leaf-size picker, and the
binding's argument checks that fire before any device call."""
import numpy as np
import pytest

from paper_1709_05061_gb300 import tune
from paper_1709_05061_gb300 import workloads as W


def test_log_uniform_ints_bounds_and_spread():
    rng = np.random.Generator(np.random.PCG64(0))
    x = W.log_uniform_ints(rng, 64, 1 << 18, 20000)
    assert x.min() >= 64 and x.max() <= 1 << 18
    # log-uniform: each of the 12 octaves holds about 1/12 of the draws
    oct_ = np.floor(np.log2(x) - 6).astype(int).clip(0, 11)
    frac = np.bincount(oct_, minlength=12) / x.size
    assert np.all(np.abs(frac - 1 / 12) < 0.02), frac


def test_many_graph_workload_promises():
    a = W.ManyGraphWorkload(8, 1 << 10, 1 << 14, 64, 1 << 12, steps=3, seed=2)
    b = W.ManyGraphWorkload(8, 1 << 10, 1 << 14, 64, 1 << 12, steps=3, seed=2)
    assert np.array_equal(a.edges, b.edges) and np.array_equal(a.batch, b.batch)
    assert np.all(a.batch <= a.edges) and np.all(a.batch % 2 == 0)
    live = [set(w.initial.tolist()) for w in a.windows]
    for i, w in enumerate(a.windows):
        assert np.array_equal(w.initial, b.windows[i].initial)
        assert len(live[i]) == a.edges[i]
        assert np.unique(w.stream).size == w.stream.size
        src, dst = W.split_keys(w.stream)
        assert np.all(src != dst) and src.max() < a.n_vertices(i) and dst.max() < a.n_vertices(i)
    for _ in range(a.steps):
        for i, (ins, dels) in enumerate(a.slide()):
            assert ins.size == dels.size == a.batch[i] // 2
            assert set(dels.tolist()) <= live[i] and not (set(ins.tolist()) & live[i])
            live[i] = (live[i] - set(dels.tolist())) | set(ins.tolist())
            assert len(live[i]) == a.edges[i]


def test_pick_leaf_size():
    assert tune.pick_leaf_size({32: 0.5, 64: 0.3, 128: 0.4}) == 64
    assert tune.pick_leaf_size({256: 0.3, 64: 0.3, 1024: 0.9}) == 64  # tie: smaller L
    for bad in ({}, {48: 1.0}, {2048: 1.0}, {1: 1.0}):
        with pytest.raises(ValueError):
            tune.pick_leaf_size(bad)
    assert all(L & (L - 1) == 0 for L in tune.LEAF_CANDIDATES)
