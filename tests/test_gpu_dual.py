"""Dual (non-lazy) deletion on the GPU against the oracle: the hand-computed cases,
random streams that grow and then shrink the array (stats and layout per batch,
with stats and on the replayed-graph path without them), and sliding windows
with analytics."""
import numpy as np
import pytest

import oracle
from helpers import apply_set_semantics, ints, parse_leaves, read_golden

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1709_05061_gb300 as gp  # noqa: E402
from paper_1709_05061_gb300 import workloads as W  # noqa: E402
from test_gpu_parity import STAT_KEYS, compare_graph, compare_layout, dev, host  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    gp.build()
    gp.lib()


@pytest.mark.parametrize("case", ["d1", "d2", "d3", "d4"])
def test_dual_worked_examples(case):
    g_ = read_golden("dual_w.txt")
    L = int(g_["L"])
    init = parse_leaves(g_["initial"], L)
    g = gp.Graph(0, leaf_size=L, raw_keys=True, dual=True, tau0=92, tauh=80, rho0=8, rhoh=40)
    g.import_layout(dev(init))
    o = oracle.OraclePMA(0, L=L, raw_keys=True, dual=True)
    o.import_layout(init)
    ins, dels = ints(g_[f"{case}_insert"]), ints(g_[f"{case}_delete"])
    st = g.update(dev(ins) if ins else None, dev(dels), stats=True)
    rc, so = o.update(ins, dels)
    assert rc == 0
    for k in STAT_KEYS:
        assert st[k] == so[k], (k, st[k], so[k])
    assert g.capacity == int(g_[f"{case}_capacity"])
    assert np.array_equal(host(g.layout()), parse_leaves(g_[f"{case}_final"], L))
    compare_layout(g, o)


def _random_batch(rng, V, live, n):
    live_l = np.array(sorted(live), np.uint64)
    ins = W.make_keys(rng.integers(0, V, n), rng.integers(0, V, n))
    ins = ins[(ins >> np.uint64(32)) != (ins & np.uint64(0xFFFFFFFF))]
    dels = live_l[rng.integers(0, live_l.size, n)] if live_l.size else np.zeros(0, np.uint64)
    extra = W.make_keys(rng.integers(0, V, n // 4), rng.integers(0, V, n // 4))
    return ins, np.concatenate([dels, extra, ins[: n // 8]])


@pytest.mark.parametrize("V,L,seed,stats", [(60, 4, 1, True), (400, 8, 2, True), (3000, 64, 3, True),
                                            (1500, 16, 4, True), (3000, 64, 5, False), (700, 32, 6, False)])
def test_dual_grow_then_shrink(V, L, seed, stats):
    rng = np.random.default_rng(seed)
    g = gp.Graph(V, leaf_size=L, dual=True)
    o = oracle.OraclePMA(V, L=L, dual=True)
    live, shrinks = set(), 0
    for it in range(36):
        n = int(rng.integers(1, 3 * V))
        ins, dels = _random_batch(rng, V, live, n)
        if it >= 14 and it % 6:  # mostly deletes: the window empties and the array shrinks
            ins = ins[: ins.size // 10]
            dels = np.concatenate([dels, np.array(sorted(live), np.uint64)[::2]])
        cap = g.capacity
        if stats:
            st = g.update(dev(ins), dev(dels), stats=True)
            rc, so = o.update(ins, dels)
            assert rc == 0
            for k in STAT_KEYS:
                assert st[k] == so[k], (it, k, st[k], so[k])
            shrinks += st["resized"] == 2
        else:
            g.update(dev(ins), dev(dels))
            assert o.update(ins, dels)[0] == 0
            shrinks += g.capacity < cap
        live = apply_set_semantics(live, ins, dels)
        compare_layout(g, o)
    g.status()
    assert shrinks >= 1
    assert g.num_edges() == len(live)


def test_dual_sliding_window_with_analytics():
    V, E0, B = 1024, 8192, 256
    stream = W.er_stream(V, E0 + 12 * B, seed=0)
    win = W.SlidingWindow(stream, E0)
    g = gp.Graph(V, leaf_size=64, dual=True)
    o = oracle.OraclePMA(V, L=64, dual=True)
    g.update(dev(win.initial), None, stats=True)
    o.update(win.initial)
    compare_graph(g, o)
    for _ in range(12):
        ins, dels = win.slide(B)
        st = g.update(dev(ins), dev(dels), stats=True)
        rc, so = o.update(ins, dels)
        for k in STAT_KEYS:
            assert st[k] == so[k], (k, st[k], so[k])
    compare_graph(g, o, srcs=(0, 17))


def test_dual_rmat_window_no_stats():
    scale, window = 14, 200_000
    stream = W.rmat_stream(scale, window + 20 * 5000, seed=3)
    win = W.SlidingWindow(stream, window)
    V = 1 << scale
    g = gp.Graph(V, leaf_size=64, dual=True)
    o = oracle.OraclePMA(V, L=64, dual=True)
    g.update(dev(win.initial))
    o.update(win.initial)
    for k in range(20):
        ins, dels = win.slide(5000 if k % 2 else 40)
        g.update(dev(ins), dev(dels))
        o.update(ins, dels)
    g.status()
    compare_layout(g, o)
