"""Host-side logic that needs no GPU: the synthetic workloads' promises (seeded,
no repeats, windows slide over live edges), the leaf-size picker, and the
binding's argument checks that fire before any device call."""
import os

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
    assert tune.pick_warps({1: 0.5, 2: 0.3, 4: 0.4, 8: 0.6}) == 2
    assert tune.pick_warps({2: 0.3, 8: 0.3}) == 8  # tie: more warps
    with pytest.raises(ValueError):
        tune.pick_warps({3: 0.1})
    with pytest.raises(ValueError):
        tune.pick_warps({})


def _req(rid, kind, t, n=0):
    from paper_1709_05061_gb300 import serve as S
    k = np.arange(n, dtype=np.uint64)
    return S.Request(rid, kind, t, ins=k if kind == S.UPDATE else None, dels=k if kind == S.UPDATE else None)


def test_admit_order_coalescing_and_budget():
    from paper_1709_05061_gb300 import serve as S
    q = [_req(0, S.UPDATE, 0.0, 10), _req(1, S.UPDATE, 0.1, 10), _req(2, S.UPDATE, 0.2, 50),
         _req(3, S.BFS, 0.3), _req(4, S.UPDATE, 0.4, 5), _req(5, S.CC, 0.5)]
    # nothing has arrived yet
    assert S.admit(q, 0, -1.0, 100) == (None, 0)
    # at t=0.15 the first two updates coalesce (40 keys), the third has not arrived
    op, h = S.admit(q, 0, 0.15, 100)
    assert op.kind == S.UPDATE and [r.rid for r in op.reqs] == [0, 1] and h == 2
    # budget: 20 + 20 + 100 keys > 100 stops before request 2, which then goes alone
    op, h = S.admit(q, 0, 1.0, 100)
    assert [r.rid for r in op.reqs] == [0, 1] and h == 2
    op, h = S.admit(q, h, 1.0, 100)
    assert [r.rid for r in op.reqs] == [2] and h == 3
    # a query is never coalesced and never overtaken by a later update
    op, h = S.admit(q, h, 1.0, 100)
    assert op.kind == S.BFS and [r.rid for r in op.reqs] == [3] and h == 4
    op, h = S.admit(q, h, 1.0, 100)
    assert [r.rid for r in op.reqs] == [4] and h == 5
    op, h = S.admit(q, h, 1.0, 100)
    assert op.kind == S.CC and h == 6
    assert S.admit(q, h, 1.0, 100) == (None, 6)
    # one request larger than the budget still goes; coalescing can be turned off
    op, h = S.admit([_req(0, S.UPDATE, 0.0, 500)], 0, 1.0, 100)
    assert len(op.reqs) == 1 and h == 1
    op, h = S.admit(q, 0, 1.0, 100, coalesce=False)
    assert [r.rid for r in op.reqs] == [0] and h == 1


def test_make_requests_mix_and_arrivals():
    from paper_1709_05061_gb300 import serve as S
    stream = W.er_stream(500, 40_000, seed=3)
    win = W.SlidingWindow(stream, 10_000)
    reqs = S.make_requests(400, 500, win, rate=1000.0, seed=5, upd_lo=10, upd_hi=200)
    kinds = [r.kind for r in reqs]
    n_upd = kinds.count(S.UPDATE)
    assert 0.72 < n_upd / len(reqs) < 0.88  # 4:1
    assert all(kinds.count(k) > 10 for k in (S.BFS, S.CC, S.PAGERANK))
    t = np.array([r.arrival for r in reqs])
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)
    assert 0.3 < t[-1] < 0.5  # 400 arrivals at 1000/s
    live = set(win.initial.tolist())
    for r in reqs:
        if r.kind == S.UPDATE:
            assert 5 <= r.ins.size <= 100 and r.ins.size == r.dels.size
            assert set(r.dels.tolist()) <= live and not (set(r.ins.tolist()) & live)
            live = (live - set(r.dels.tolist())) | set(r.ins.tolist())
        else:
            assert 0 <= r.src < 500


def test_serve_budget_split():
    from paper_1709_05061_gb300 import serve as S
    # 1 GiB: 512 MiB for keys (two buffers of 8-byte keys, capped) and 512 MiB of 64 MiB results (capped at 8)
    keys, slots = S.Server.budget_split(1 << 30, 1 << 24)
    assert keys == 1 << 22 and slots == 8
    keys, slots = S.Server.budget_split(100 << 20, 1 << 24)  # 50 MiB each side
    assert keys == (50 << 20) // 16 and slots == 1
    assert 2 * 8 * keys + 4 * (1 << 24) * slots <= (100 << 20) + 4 * (1 << 24)  # at least one slot always
    keys, slots = S.Server.budget_split(0, 10)
    assert keys == 1024 and slots == 1


def test_clock_summary_keeps_samples_of_the_timed_region():
    """bench.py's clock record: only samples taken between the start and the end of
    the timed region, plus the first one after it, count; a throttle reason seen
    outside that window is not reported."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    c = bench.ClockSampler(0)
    row = "0, {sm}, 2070, 900.0, 0x0, Not Active, Not Active, {thermal}, Not Active"
    c.lines = [(0.5, row.format(sm=1200, thermal="Active")),   # before the region
               (1.1, row.format(sm=2070, thermal="Not Active")),
               (1.2, row.format(sm=2060, thermal="Not Active")),
               (2.1, row.format(sm=2070, thermal="Not Active")),  # first one after
               (2.2, row.format(sm=900, thermal="Active"))]
    c.t0, c.t1 = 1.0, 2.0
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2070 and s["reasons"] == []
    c.lines = []
    assert c.summary()["reasons"] == ["unsampled"]
