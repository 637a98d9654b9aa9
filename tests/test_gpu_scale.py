"""Parity at full size: the R-MAT scale-20 sliding window that bench.py times
(2^20 vertices, 16,000,000-edge window, leaf size 64), bulk load plus batches of
10^2, 10^4 and 10^6 updates, through the same library calls as the benchmark.
The oracle computes the whole array, so the layout is compared slot for slot
(33.5M slots); BFS, CC and PageRank are compared in full."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1709_05061_gb300 as gp  # noqa: E402
from paper_1709_05061_gb300 import workloads as W  # noqa: E402

STATS = ("n_inserted", "n_deleted", "n_ignored", "levels_climbed", "resized", "alg_bytes", "touched_leaves",
         "covered_leaves", "merges", "delete_leaves")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def test_rmat20_window_full_size():
    gp.build()
    scale, window = 20, 16_000_000
    batches = (100, 10_000, 1_000_000)
    stream = W.rmat_stream(scale, window + sum(b // 2 for b in batches), seed=1, samples=1 << 24)
    win = W.SlidingWindow(stream, window)
    V = 1 << scale
    g = gp.Graph(V, leaf_size=64)
    o = oracle.OraclePMA(V, L=64)

    def step(ins, dels):
        st = g.update(dev(ins), dev(dels) if dels is not None else None, stats=True)
        rc, so = o.update(ins, dels if dels is not None else [])
        assert rc == 0
        for k in STATS:
            assert st[k] == so[k], (k, st[k], so[k])
        lg = g.layout().cpu().numpy().view(np.uint64)
        lo = o.layout()
        assert lg.size == lo.size
        bad = np.count_nonzero(lg != lo)
        assert bad == 0, f"{bad} slots differ"
        assert g.check() == 0

    step(win.initial, None)
    assert g.capacity == 1 << 25
    for b in batches:
        ins, dels = win.slide(b // 2)
        step(ins, dels)
    src = int(stream[0] >> np.uint64(32))
    assert np.array_equal(g.bfs(src).cpu().numpy(), o.bfs(src))
    assert np.array_equal(g.cc().cpu().numpy().view(np.uint32), o.cc())
    pr = g.pagerank(20, 0.85).cpu().numpy().astype(np.float64)
    ref = o.pagerank(20, 0.85)
    rel = np.max(np.abs(pr - ref) / ref)
    assert rel <= 1e-5, rel
    assert np.array_equal(g.row_end().cpu().numpy().view(np.uint32), o.row_end())


def test_chung_lu_learned_full_size():
    """The learned-search workload at full size: Chung-Lu, 1.6M vertices, 30M edges
    (degree exponent 2.1, seed 7), batches of 1e5 (70% new edges, 30% random live
    edges).  The learned and the plain search give the oracle's array slot for slot."""
    V, E0, B = 1_600_000, 30_000_000, 100_000
    n_ins, n_del = 70_000, 30_000
    stream = W.chung_lu_stream(V, E0 + 4 * n_ins, gamma=2.1, seed=7)
    rng = np.random.default_rng(7)
    live = stream[:E0].copy()
    learned, plain = gp.Graph(V, leaf_size=64), gp.Graph(V, leaf_size=64, plain_search=True)
    o = oracle.OraclePMA(V, L=64)
    for g in (learned, plain):
        g.update(dev(stream[:E0]), None)
    o.update(stream[:E0])
    for i in range(4):
        ins = stream[E0 + i * n_ins: E0 + (i + 1) * n_ins]
        pick = rng.choice(live.size, n_del, replace=False)
        dels = live[pick]
        keep = np.ones(live.size, bool)
        keep[pick] = False
        live = np.concatenate([live[keep], ins])
        for g in (learned, plain):
            g.update(dev(ins), dev(dels))
        o.update(ins, dels)
    lo = o.layout()
    for g in (learned, plain):
        g.status()
        lg = g.layout().cpu().numpy().view(np.uint64)
        assert lg.size == lo.size and np.count_nonzero(lg != lo) == 0
        assert g.check() == 0


@pytest.mark.parametrize("V", [1 << 25, (1 << 25) + 1])
def test_pagerank_largest_bucketed_graph(V):
    """2^25 vertices is the largest graph the bucketed PageRank pass takes (4096
    buckets of 8192 heads: the bucket tables of the count and placement kernels at
    their largest); one vertex more and the library takes the push pass.  Both give
    the ranks of a handle forced onto the push pass, bit for bit, on an R-MAT
    scale-25 stream of 2^22 samples held on the device."""
    gp.build()
    st = W.rmat_stream_device(25, 1 << 22, seed=5)
    a, b = gp.Graph(V, leaf_size=64), gp.Graph(V, leaf_size=64, push_pagerank=True)
    for g in (a, b):
        g.update(st)
    ra = a.pagerank(5, 0.85).cpu().numpy()
    rb = b.pagerank(5, 0.85).cpu().numpy()
    assert np.array_equal(ra.view(np.uint32), rb.view(np.uint32))
    assert abs(float(ra.astype(np.float64).sum()) - 1.0) < 1e-3
    a.status()
    b.status()


@pytest.mark.parametrize("scale", [21, 22])
def test_large_graph_analytics_match_oracle(scale):
    """Graphs past 2^20 vertices take other branches of the analytics: from 2^21
    vertices (256 head buckets of 8192) the bucketed PageRank runs one block per
    bucket, and at 2^22 (512 buckets) the placement writes every edge straight to
    its bucket.  R-MAT with 2^(scale+1) distinct edges: layout slot for
    slot, BFS from two sources and CC exactly, PageRank-20 (bucketed and push
    passes) within 1e-5 of the oracle's FP64 ranks, and the two passes bit for bit
    equal."""
    gp.build()
    V = 1 << scale
    stream = W.rmat_stream(scale, 1 << (scale + 1), seed=50 + scale)
    o = oracle.OraclePMA(V, L=64)
    assert o.update(stream)[0] == 0
    gb, gpush = gp.Graph(V, leaf_size=64), gp.Graph(V, leaf_size=64, push_pagerank=True)
    for g in (gb, gpush):
        g.update(dev(stream), None, stats=True)
    lg = gb.layout().cpu().numpy().view(np.uint64)
    lo = o.layout()
    assert lg.size == lo.size and np.count_nonzero(lg != lo) == 0
    assert gb.check() == 0
    srcs = (int(stream[0] >> np.uint64(32)), int(stream[len(stream) // 2] >> np.uint64(32)))
    for s in srcs:
        assert np.array_equal(gb.bfs(s).cpu().numpy(), o.bfs(s)), s
    assert np.array_equal(gb.cc().cpu().numpy().view(np.uint32), o.cc())
    ref = o.pagerank(20, 0.85)
    rb = gb.pagerank(20, 0.85).cpu().numpy()
    rp = gpush.pagerank(20, 0.85).cpu().numpy()
    assert np.array_equal(rb.view(np.uint32), rp.view(np.uint32))
    rel = np.max(np.abs(rb.astype(np.float64) - ref) / ref)
    assert rel <= 1e-5, rel
    for g in (gb, gpush):
        g.status()
        g.close()
