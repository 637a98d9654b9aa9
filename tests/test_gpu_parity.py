"""GPU parity: the CUDA library against the CPU oracle, element by element,
through the C ABI (via the thin binding).  Layout, exported edges, CSR, guard
index, stats: bit-exact.  BFS depths and CC labels: exact.  PageRank (FP32):
max relative error <= 1e-5 against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from helpers import EMPTY, apply_set_semantics, ints, parse_leaves, read_golden

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1709_05061_gb300 as gp  # noqa: E402
from paper_1709_05061_gb300 import workloads as W  # noqa: E402

PR_TOL = 1e-5
STAT_KEYS = ("n_inserted", "n_deleted", "n_ignored", "levels_climbed", "resized", "alg_bytes",
             "touched_leaves", "covered_leaves", "merges", "delete_leaves")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.uint64)).view(np.int64)).cuda()


def host(t):
    return t.cpu().numpy().view(np.uint64)


@pytest.fixture(scope="module", autouse=True)
def built():
    gp.build()
    gp.lib()


def compare_layout(g, o):
    lg, lo = host(g.layout()), o.layout()
    assert lg.size == lo.size, (lg.size, lo.size)
    bad = np.nonzero(lg != lo)[0]
    assert bad.size == 0, f"layout differs at {bad.size} slots, first {bad[:8]}: gpu {lg[bad[:4]]} oracle {lo[bad[:4]]}"
    assert g.check() == 0, f"device checker code {g.check()}"


def compare_graph(g, o, srcs=(0,), pr_iters=20):
    compare_layout(g, o)
    assert np.array_equal(g.row_end().cpu().numpy().view(np.uint32), o.row_end())
    assert np.array_equal(host(g.export_sorted()), o.export_sorted())
    rp, col = g.export_csr()
    orp, ocol = o.export_csr()
    assert np.array_equal(rp.cpu().numpy().view(np.uint64), orp)
    assert np.array_equal(col.cpu().numpy().view(np.uint32), ocol)
    for s in srcs:
        assert np.array_equal(g.bfs(s).cpu().numpy(), o.bfs(s))
    assert np.array_equal(g.cc().cpu().numpy().view(np.uint32), o.cc())
    pr = g.pagerank(pr_iters, 0.85).cpu().numpy().astype(np.float64)
    ref = o.pagerank(pr_iters, 0.85)
    rel = np.max(np.abs(pr - ref) / ref)
    assert rel <= PR_TOL, rel


def both_update(g, o, ins, dels):
    st = g.update(dev(ins) if ins is not None else None, dev(dels) if dels is not None else None, stats=True)
    rc, so = o.update(ins if ins is not None else [], dels if dels is not None else [])
    assert rc == 0
    for k in STAT_KEYS:
        assert st[k] == so[k], (k, st[k], so[k])
    return st


# ---- the tiny configuration: ER 1,024 vertices, 8,192 edges, 16 slides of 256 --------------
def test_er_1024_sliding_window():
    V, E0, B = 1024, 8192, 256
    stream = W.er_stream(V, E0 + 16 * B, seed=0)
    win = W.SlidingWindow(stream, E0)
    g = gp.Graph(V, leaf_size=64)
    o = oracle.OraclePMA(V, L=64)
    compare_graph(g, o)
    both_update(g, o, win.initial, None)
    compare_graph(g, o)
    assert g.capacity == 16384
    for b in range(16):
        ins, dels = win.slide(B)
        both_update(g, o, ins, dels)
        compare_graph(g, o, srcs=(0, int(b * 61 % V)))
        assert g.num_edges() == E0


# ---- the paper's worked examples on the GPU ---------------------------------------------------
@pytest.mark.parametrize("ex", ["ex3", "ex1"])
def test_worked_examples_gpu(ex):
    gd = read_golden("example_w.txt")
    L = int(gd["L"])
    init = parse_leaves(gd["initial"], L)
    g = gp.Graph(0, leaf_size=L, raw_keys=True)
    g.import_layout(dev(init))
    assert np.array_equal(host(g.layout()), init)
    st = g.update(dev(ints(gd[f"{ex}_insert"])), None, stats=True)
    assert np.array_equal(host(g.layout()), parse_leaves(gd[f"{ex}_final"], L))
    assert st["merges"][:4] == ints(gd[f"{ex}_merges_per_level"])
    assert g.check() == 0


# ---- randomized batches of every composition, several leaf sizes ------------------------------
def random_batch(rng, V, live, n):
    live_l = list(live)
    ins = [(int(a) << 32) | int(b) for a, b in rng.integers(0, V, (n, 2))]
    if live_l:
        ins += [live_l[i] for i in rng.integers(0, len(live_l), n // 4)]
    ins += ins[: n // 8]
    dels = [live_l[i] for i in rng.integers(0, len(live_l), n)] if live_l else []
    dels += [(int(a) << 32) | int(b) for a, b in rng.integers(0, V, (n // 4, 2))]
    dels += ins[: n // 8]
    return (rng.permutation(np.array(ins, np.uint64)) if ins else np.zeros(0, np.uint64),
            rng.permutation(np.array(dels, np.uint64)) if dels else np.zeros(0, np.uint64))


@pytest.mark.parametrize("V,L,seed", [(40, 4, 0), (200, 8, 1), (300, 32, 2), (1000, 64, 3), (3000, 128, 4),
                                      (2000, 256, 5), (5000, 1024, 6), (700, 2, 7)])
def test_random_batches(V, L, seed):
    rng = np.random.default_rng(seed)
    g = gp.Graph(V, leaf_size=L)
    o = oracle.OraclePMA(V, L=L)
    compare_layout(g, o)
    live = set()
    for it in range(24):
        n = int(rng.integers(0, 3 * V if it % 5 else 10 * V))
        ins, dels = random_batch(rng, V, live, n)
        both_update(g, o, ins, dels)
        live = apply_set_semantics(live, ins, dels)
        compare_layout(g, o)
    compare_graph(g, o, srcs=(0, V - 1))


def test_raw_keys_random_layouts():
    rng = np.random.default_rng(9)
    for L in (4, 16, 64):
        g = gp.Graph(0, leaf_size=L, raw_keys=True)
        o = oracle.OraclePMA(0, L=L, raw_keys=True)
        live = set()
        for it in range(20):
            k = rng.integers(0, 1 << 62, 400, dtype=np.int64).astype(np.uint64) % np.uint64(5000)
            ins = k[:300]
            dels = np.array(list(live)[: 100] if live else [], np.uint64)
            both_update(g, o, ins, dels)
            live = apply_set_semantics(live, ins, dels)
            compare_layout(g, o)


# ---- edge cases -------------------------------------------------------------------------------
def test_edge_cases():
    V, L = 500, 64
    g = gp.Graph(V, leaf_size=L)
    o = oracle.OraclePMA(V, L=L)
    rng = np.random.default_rng(1)
    base = W.er_stream(V, 4000, seed=3)
    both_update(g, o, base, None)
    compare_graph(g, o, srcs=(0, V - 1))
    # empty batch
    st = g.update(None, None, stats=True)
    assert st["n_inserted"] == 0 and st["n_ignored"] == 0
    # only deletes, with duplicates and absent keys
    d = np.concatenate([base[:300], base[:50], W.make_keys(np.arange(10), np.arange(10) + 1)])
    both_update(g, o, None, d)
    compare_layout(g, o)
    # insert and delete of the same keys cancel; re-inserting stored keys is ignored
    both_update(g, o, base[300:400], base[300:400])
    both_update(g, o, base[400:500], None)
    compare_layout(g, o)
    # keys at vertex 0 and V-1, self-loops
    ek = W.make_keys(np.array([0, 0, V - 1, V - 1, 7]), np.array([V - 1, 0, 0, V - 1, 7]))
    both_update(g, o, ek, None)
    compare_graph(g, o, srcs=(0, V - 1, 7))
    # one hot vertex: many inserts into one row (escalates far above its leaf)
    hot = W.make_keys(np.full(V, 3), np.arange(V))
    both_update(g, o, hot, None)
    compare_graph(g, o, srcs=(3,))
    # sorted and reverse-sorted batches
    s2 = np.sort(W.er_stream(V, 3000, seed=11))
    both_update(g, o, s2[:1500], None)
    both_update(g, o, s2[1500:][::-1].copy(), s2[:700][::-1].copy())
    compare_graph(g, o, srcs=(0, 100))
    # a batch that forces the capacity to grow
    cap0 = g.capacity
    big = W.er_stream(V, 60000, seed=12)
    st = both_update(g, o, big, None)
    assert st["resized"] == 1 and g.capacity > cap0
    compare_graph(g, o, srcs=(0,))
    # delete everything but the guards
    live = o.export_sorted()
    both_update(g, o, None, rng.permutation(live))
    compare_graph(g, o, srcs=(0,))
    assert g.num_edges() == 0


def test_invalid_keys_change_nothing():
    V = 100
    g = gp.Graph(V, leaf_size=8)
    g.update(dev(W.er_stream(V, 500, seed=4)), None, stats=True)
    before = host(g.layout())
    for bad in ([V << 32 | 1], [1 << 32 | V], [(1 << 32) | 0xFFFFFFFF]):
        with pytest.raises(gp.GpmaError) as e:
            g.update(dev([(2 << 32) | 3] + bad), None, stats=True)
        assert e.value.code == gp.GPMA_EINVAL
        assert np.array_equal(host(g.layout()), before)
    with pytest.raises(gp.GpmaError):
        g.update(None, dev([(5 << 32) | 0xFFFFFFFF]), stats=True)
    # without stats the error surfaces at the next status call and nothing is applied
    g.update(dev([(2 << 32) | 3, V << 32]), None)
    with pytest.raises(gp.GpmaError):
        g.status()
    g.status()  # cleared
    assert np.array_equal(host(g.layout()), before)
    assert g.check() == 0


def test_async_batches_then_status():
    V = 2048
    stream = W.rmat_stream(11, 20000 + 20 * 500, seed=5)
    win = W.SlidingWindow(stream, 20000)
    g = gp.Graph(V, leaf_size=64)
    o = oracle.OraclePMA(V, L=64)
    g.update(dev(win.initial), None)
    o.update(win.initial)
    for _ in range(20):
        ins, dels = win.slide(500)
        g.update(dev(ins), dev(dels))
        o.update(ins, dels)
    g.status()
    compare_graph(g, o, srcs=(int(W.split_keys(stream[:1])[0][0]),))


def test_export_capacity_errors():
    g = gp.Graph(50, leaf_size=8)
    g.update(dev(W.er_stream(50, 300, seed=1)), None, stats=True)
    small = torch.empty(10, dtype=torch.int64, device="cuda")
    assert gp.gpma_export_sorted(g.h, small) == -301
    assert gp.gpma_export_layout(g.h, small) < 0


def test_import_rejects_bad_layouts():
    g = gp.Graph(0, leaf_size=4, raw_keys=True)
    good = parse_leaves(read_golden("example_w.txt")["initial"], 4)
    g.import_layout(dev(good))
    bad = good.copy()
    bad[0], bad[4] = bad[4], bad[0]  # order broken
    with pytest.raises(gp.GpmaError):
        g.import_layout(dev(bad))
    assert np.array_equal(host(g.layout()), good)
    with pytest.raises(gp.GpmaError):
        g.import_layout(dev(good[:12]))  # not L * 2^k


# ---- learned leaf search: the same array as plain binary search ----------------------------------
def test_learned_search_matches_plain():
    rng = np.random.default_rng(17)
    scale = 14
    V = 1 << scale
    stream = W.rmat_stream(scale, 400_000, seed=8)
    learned = gp.Graph(V, leaf_size=64)
    plain = gp.Graph(V, leaf_size=64, plain_search=True)
    o = oracle.OraclePMA(V, L=64)
    win = W.SlidingWindow(stream, 100_000)
    for g in (learned, plain):
        g.update(dev(win.initial), None, stats=True)
    o.update(win.initial)
    # growth (escalations, resizes) then sliding batches of mixed sizes
    for step in range(40):
        b = int(rng.choice([64, 1000, 5000, 20000]))
        if step < 8:
            ins, dels = win.stream[win.tail: win.tail + b], np.zeros(0, np.uint64)
            win.tail += b
        else:
            ins, dels = win.slide(b // 2)
        st1 = learned.update(dev(ins), dev(dels) if dels.size else None, stats=True)
        st2 = plain.update(dev(ins), dev(dels) if dels.size else None, stats=True)
        o.update(ins, dels)
        assert st2["model_sorted"] == 0  # which sort ran may differ; everything else may not
        st1.pop("model_sorted")
        st2.pop("model_sorted")
        assert st1 == st2
        a, b2 = host(learned.layout()), host(plain.layout())
        assert np.array_equal(a, b2), f"step {step}: learned and plain layouts differ"
    assert np.array_equal(host(learned.layout()), o.layout())
    assert learned.check() == 0


def test_growth_without_stats_matches_oracle():
    """Insert-only batches of about a tenth of the array, no stats: batches that
    may overflow the root replay the graph that grows the array on the device
    (into the spare of height h+1); layout and capacity follow the oracle."""
    V = 4096
    stream = W.er_stream(V, 120_000, seed=21)
    g = gp.Graph(V, leaf_size=32)
    o = oracle.OraclePMA(V, L=32)
    caps = set()
    at = 0
    while at < stream.size:
        k = max(256, (V + at) // 10)
        ins = stream[at: at + k]
        at += k
        g.update(dev(ins), None)
        o.update(ins)
        lg = host(g.layout())
        lo = o.layout()
        assert lg.size == lo.size == g.capacity
        assert np.array_equal(lg, lo)
        caps.add(g.capacity)
    g.status()
    assert len(caps) >= 4
    assert g.check() == 0
    assert g.num_edges() == stream.size


def test_pagerank_mid_size():
    """R-MAT scale 16, 10^6 edges (2^21 slots): ranks after 1 and 20 iterations,
    BFS and CC against the oracle."""
    V = 1 << 16
    stream = W.rmat_stream(16, 1_000_000, seed=8)
    g = gp.Graph(V, leaf_size=64)
    o = oracle.OraclePMA(V, L=64)
    g.update(dev(stream), None, stats=True)
    o.update(stream)
    assert g.capacity == 1 << 21
    for it in (1, 20):
        pr = g.pagerank(it, 0.85).cpu().numpy().astype(np.float64)
        ref = o.pagerank(it, 0.85)
        assert np.max(np.abs(pr - ref) / ref) <= PR_TOL
    g.status()
    src = int(stream[0] >> np.uint64(32))
    assert np.array_equal(g.bfs(src).cpu().numpy(), o.bfs(src))
    assert np.array_equal(g.cc().cpu().numpy().view(np.uint32), o.cc())


@pytest.mark.parametrize("V,n_edges,seed", [(1 << 16, 1_000_000, 8), (1 << 19, 1_000_000, 9), (5000, 60_000, 3),
                                            (4097, 20_000, 4), (1, 0, 0), (300, 0, 0)])
def test_pagerank_bucketed_equals_push(V, n_edges, seed):
    """The bucketed sum pass (edges copied into head buckets of 8192, partial sums
    in shared memory) and the push pass (one L2 reduction per stored edge) add the
    same fixed-point contributions, so their ranks agree bit for bit: on R-MAT
    graphs with heavy heads (8 buckets summed by clusters of 8 blocks, and 64 buckets
    by clusters of 4), on vertex counts that leave a ragged last bucket, and on
    graphs without edges.  Both stay within the tolerance of the oracle."""
    if n_edges:
        scale = max(1, int(np.ceil(np.log2(V))))
        stream = W.rmat_stream(scale, n_edges, seed=seed)
        stream = stream[((stream >> np.uint64(32)) < V) & ((stream & np.uint64(0xFFFFFFFF)) < V)]
    else:
        stream = np.zeros(0, dtype=np.uint64)
    gb = gp.Graph(V, leaf_size=64)
    gpush = gp.Graph(V, leaf_size=64, push_pagerank=True)
    o = oracle.OraclePMA(V, L=64)
    for g in (gb, gpush):
        g.update(dev(stream), None)
    o.update(stream)
    for it in (0, 1, 3, 20):
        a = gb.pagerank(it, 0.85).cpu().numpy()
        b = gpush.pagerank(it, 0.85).cpu().numpy()
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32)), it
        ref = o.pagerank(it, 0.85)
        assert np.max(np.abs(a.astype(np.float64) - ref) / ref) <= PR_TOL
    # after an update that grows the array, the edge copy is rebuilt at the new size
    if n_edges:
        more = W.rmat_stream(max(1, int(np.ceil(np.log2(V)))), 3 * n_edges, seed=seed + 100)
        more = more[((more >> np.uint64(32)) < V) & ((more & np.uint64(0xFFFFFFFF)) < V)]
        for g in (gb, gpush):
            g.update(dev(more), None)
        o.update(more)
        a = gb.pagerank(20, 0.85).cpu().numpy()
        b = gpush.pagerank(20, 0.85).cpu().numpy()
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
        ref = o.pagerank(20, 0.85)
        assert np.max(np.abs(a.astype(np.float64) - ref) / ref) <= PR_TOL
    gb.status()
    gpush.status()


def test_pagerank_snapshot_holds_the_graph_it_was_taken_on():
    """gpma_pagerank_snapshot copies the edges and out-degrees of the graph as it is
    at that point of the stream; gpma_pagerank_run then iterates over the copy.
    Updates between the two (here: inserts that grow the array, then deletes of a
    third of the edges) do not change the ranks, which equal those of one
    gpma_pagerank call on the earlier graph bit for bit and the oracle's within the
    tolerance.  A second run over the same snapshot repeats the ranks; a handle that
    sums by the push pass takes no snapshot; a run with no snapshot is refused."""
    V = 1 << 15
    stream = W.rmat_stream(15, 400_000, seed=71)
    first, more = stream[:150_000], stream[150_000:]
    g = gp.Graph(V, leaf_size=64)
    o = oracle.OraclePMA(V, L=64)
    out = torch.empty(V, dtype=torch.float32, device="cuda")
    with pytest.raises(gp.GpmaError) as e:
        gp.gpma_pagerank_run(g.h, 5, 0.85, out)
    assert e.value.code == gp.GPMA_EINVAL
    g.update(dev(first), None)
    o.update(first)
    alone = g.pagerank(20, 0.85).clone()
    ref = o.pagerank(20, 0.85)
    assert gp.gpma_pagerank_snapshot(g.h)
    cap0 = g.capacity
    g.update(dev(more), None)
    g.update(None, dev(first[::3]))
    assert g.capacity > cap0
    gp.gpma_pagerank_run(g.h, 20, 0.85, out)
    assert torch.equal(out.view(torch.int32), alone.view(torch.int32))
    assert np.max(np.abs(out.cpu().numpy().astype(np.float64) - ref) / ref) <= PR_TOL
    out2 = torch.empty_like(out)
    gp.gpma_pagerank_run(g.h, 20, 0.85, out2)
    assert torch.equal(out2.view(torch.int32), out.view(torch.int32))
    # a new snapshot sees the updates
    o.update(more)
    o.update(np.zeros(0, np.uint64), first[::3])
    assert gp.gpma_pagerank_snapshot(g.h)
    gp.gpma_pagerank_run(g.h, 20, 0.85, out)
    assert torch.equal(out.view(torch.int32), g.pagerank(20, 0.85).view(torch.int32))
    ref2 = o.pagerank(20, 0.85)
    assert np.max(np.abs(out.cpu().numpy().astype(np.float64) - ref2) / ref2) <= PR_TOL
    g.status()
    g.close()
    gpush = gp.Graph(V, leaf_size=64, push_pagerank=True)
    gpush.update(dev(first), None)
    assert not gp.gpma_pagerank_snapshot(gpush.h)
    with pytest.raises(gp.GpmaError) as e:
        gp.gpma_pagerank_run(gpush.h, 5, 0.85, out)
    assert e.value.code == gp.GPMA_EINVAL
    gpush.status()
    gpush.close()
