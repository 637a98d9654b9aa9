"""Batched many-graph update: gpma_update_many against per-graph sequential GPU
runs and the oracle, slot for slot, on R-MAT sliding windows of uneven sizes
(edge counts and batch sizes log-uniform), at the fixed leaf size and at the
leaf size and warps per leaf-pass block the autotuner picks."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1709_05061_gb300 as gp  # noqa: E402
from paper_1709_05061_gb300 import tune  # noqa: E402
from paper_1709_05061_gb300 import workloads as W  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.uint64)).view(np.int64)).cuda()


def host(t):
    return t.cpu().numpy().view(np.uint64)


def run_many(wl, leaf_sizes, check_oracle=True, leaf_warps=None):
    n = wl.n_graphs
    wpb = leaf_warps or [0] * n
    many = [gp.Graph(wl.n_vertices(i), leaf_size=leaf_sizes[i], leaf_warps=wpb[i]) for i in range(n)]
    seq = [gp.Graph(wl.n_vertices(i), leaf_size=leaf_sizes[i], leaf_warps=wpb[i]) for i in range(n)]
    orc = [oracle.OraclePMA(wl.n_vertices(i), L=leaf_sizes[i]) for i in range(n)] if check_oracle else []
    init = [dev(w.initial) for w in wl.windows]
    gp.Graph.update_many(many, init, [None] * n)
    for i in range(n):
        seq[i].update(init[i])
        if orc:
            orc[i].update(wl.windows[i].initial)
    for _ in range(wl.steps):
        batch = wl.slide()
        ins = [dev(b[0]) for b in batch]
        dels = [dev(b[1]) for b in batch]
        gp.Graph.update_many(many, ins, dels)
        for i in range(n):
            seq[i].update(ins[i], dels[i])
            if orc:
                assert orc[i].update(batch[i][0], batch[i][1])[0] == 0
    torch.cuda.synchronize()
    for i in range(n):
        many[i].status()
        lm = host(many[i].layout())
        assert np.array_equal(lm, host(seq[i].layout())), f"graph {i}: batched != sequential"
        if orc:
            lo = orc[i].layout()
            assert lm.size == lo.size and np.count_nonzero(lm != lo) == 0, f"graph {i}: batched != oracle"
        assert many[i].check() == 0
        assert many[i].num_edges() == wl.edges[i]
    return many


def test_many_uneven_graphs_match_sequential_and_oracle():
    gp.build()
    wl = W.ManyGraphWorkload(16, 1 << 10, 1 << 16, 64, 1 << 12, steps=4, seed=3)
    run_many(wl, [64] * wl.n_graphs)


def test_many_mixed_leaf_sizes():
    wl = W.ManyGraphWorkload(12, 1 << 10, 1 << 15, 64, 1 << 11, steps=3, seed=4)
    sizes = [tune.LEAF_CANDIDATES[i % len(tune.LEAF_CANDIDATES)] for i in range(wl.n_graphs)]
    run_many(wl, sizes)


def test_many_at_tuned_leaf_size():
    wl = W.ManyGraphWorkload(4, 1 << 12, 1 << 15, 256, 1 << 12, steps=3, seed=5)
    sizes, warps = [], []
    for i, w in enumerate(wl.windows):
        half = int(wl.batch[i]) // 2
        ins = w.stream[w.tail: w.tail + half]
        dels = w.stream[w.head: w.head + half]
        L, wpb, ltab, wtab = tune.autotune(wl.n_vertices(i), dev(w.initial), dev(ins), dev(dels), reps=2)
        assert set(ltab) == set(tune.LEAF_CANDIDATES) and all(t > 0 for t in ltab.values())
        assert set(wtab) == set(tune.WARP_CANDIDATES) and all(t > 0 for t in wtab.values())
        assert L == tune.pick_leaf_size(ltab) and wpb == tune.pick_warps(wtab)
        sizes.append(L)
        warps.append(wpb)
    run_many(wl, sizes, leaf_warps=warps)


def test_many_edge_cases():
    gp.gpma_update_many([], [], [])  # nothing to do
    a, b = gp.Graph(64, leaf_size=8), gp.Graph(64, leaf_size=16)
    keys = W.er_stream(64, 300, seed=9)
    with pytest.raises(gp.GpmaError) as e:
        gp.gpma_update_many([a.h, a.h], [dev(keys[:10]), dev(keys[10:20])], [None, None])
    assert e.value.code == gp.GPMA_EINVAL
    # one empty batch, one invalid batch: the invalid one changes nothing and is
    # reported by its own handle's status; the other is applied
    gp.Graph.update_many([a, b], [dev(keys[:100]), dev(keys[100:200])], [None, None])
    before_b = host(b.layout())
    bad = np.concatenate([keys[200:210], np.array([64 << 32 | 1], np.uint64)])
    gp.Graph.update_many([a, b], [None, dev(bad)], [dev(keys[:50]), None])
    a.status()
    with pytest.raises(gp.GpmaError):
        b.status()
    assert np.array_equal(host(b.layout()), before_b)
    assert a.num_edges() == 50 and b.num_edges() == 100
    assert a.check() == 0 and b.check() == 0


def test_many_batched_stages_vary_per_call():
    """One set of handles, several calls with different batch sizes (the batched
    graph is captured once; the per-call plan table sizes every launch): one-block
    and radix front ends in the same call, a batch that needs four search words a
    thread (more than 2^19 keys), leaf sizes 32..1024 with the tuned warps per
    block of the one-warp-per-leaf pass, a raw-key handle, and inserts crowded into
    a few rows so that leaves overflow and the handles' merge levels run in their
    own graph branches.  After every call each handle equals the same handle
    updated alone and the oracle, slot for slot."""
    gp.build()
    rng = np.random.default_rng(21)
    specs = [(1 << 12, 32, 0), (1 << 14, 64, 0), (1 << 15, 128, 2), (1 << 16, 256, 4), (1 << 13, 512, 1),
             (1 << 12, 1024, 8), (1 << 20, 64, 0), (1 << 14, 16, 0)]
    many, seq, orc, streams = [], [], [], []
    for i, (V, L, wpb) in enumerate(specs):
        raw = i == len(specs) - 1
        many.append(gp.Graph(V, leaf_size=L, leaf_warps=wpb, raw_keys=raw))
        seq.append(gp.Graph(V, leaf_size=L, leaf_warps=wpb, raw_keys=raw))
        orc.append(oracle.OraclePMA(V, L=L, raw_keys=raw))
        scale = int(np.log2(V))
        streams.append(W.rmat_stream(scale, (1 << 20) + 3 * 600_000 if V == 1 << 20 else 6 * V, seed=300 + i))
    wins = [W.SlidingWindow(st, len(st) // 3 if len(st) < 1 << 20 else 1 << 20) for st in streams]
    init = [dev(w.initial) for w in wins]
    gp.Graph.update_many(many, init, [None] * len(specs))
    for i in range(len(specs)):
        seq[i].update(init[i])
        assert orc[i].update(wins[i].initial)[0] == 0

    def hot_rows(i, n):
        V = specs[i][0]
        rows = rng.integers(0, V, 4, dtype=np.uint64)
        cols = rng.integers(0, V, n, dtype=np.uint64)
        k = (rows[rng.integers(0, 4, n)] << np.uint64(32)) | cols
        k = k[(k >> np.uint64(32)) != (k & np.uint64(0xFFFFFFFF))]
        return np.unique(k)

    for step, sizes in enumerate([(100, 3000, 20_000, 50, 9000, 200, 600_000, 700),
                                  (5000, 64, 4096, 4097, 300, 10_000, 2000, 8000),
                                  (2, 20_000, 128, 30_000, 6000, 4000, 100_000, 50)]):
        ins_l, del_l = [], []
        for i, b in enumerate(sizes):
            ins, dels = wins[i].slide(max(1, b // 2))
            if step == 1 and i in (1, 2, 3):  # crowded rows: leaves overflow, merge levels run
                extra = hot_rows(i, 3000)
                ins = np.unique(np.concatenate([ins, extra]))
            ins_l.append(ins)
            del_l.append(dels)
        gp.Graph.update_many(many, [dev(x) for x in ins_l], [dev(x) for x in del_l])
        for i in range(len(specs)):
            seq[i].update(dev(ins_l[i]), dev(del_l[i]))
            assert orc[i].update(ins_l[i], del_l[i])[0] == 0
        torch.cuda.synchronize()
        for i in range(len(specs)):
            many[i].status()
            lm = host(many[i].layout())
            assert np.array_equal(lm, host(seq[i].layout())), f"step {step} graph {i}: batched != alone"
            lo = orc[i].layout()
            assert lm.size == lo.size and np.count_nonzero(lm != lo) == 0, f"step {step} graph {i}: != oracle"
            assert many[i].check() == 0
    for g in many + seq:
        g.close()


def test_many_full_size_graphs():
    """64 graphs, edges log-uniform in [2^10, 2^22], batches log-uniform in
    [64, 2^18]: batched equals sequential and the oracle for every graph."""
    wl = W.ManyGraphWorkload(64, 1 << 10, 1 << 22, 64, 1 << 18, steps=2, seed=11)
    run_many(wl, [64] * wl.n_graphs)
