"""Served stream: every query answered inside the mix (coalesced update batches,
two streams, bounded result slots) equals the same query run alone on the same
prefix of the stream, with the updates applied one request at a time: exact for
BFS and CC, within 1e-5 relative for PageRank.  The final edge set is checked
against the oracle."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1709_05061_gb300 as gp  # noqa: E402
from paper_1709_05061_gb300 import serve as S  # noqa: E402
from paper_1709_05061_gb300 import workloads as W  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.uint64)).view(np.int64)).cuda()


def replay_alone(V, initial, reqs, L=64):
    g = gp.Graph(V, leaf_size=L)
    g.update(dev(initial))
    for r in reqs:
        if r.kind == S.UPDATE:
            g.update(dev(r.ins), dev(r.dels))
            continue
        if r.kind == S.BFS:
            alone = g.bfs(r.src).cpu().numpy()
            assert np.array_equal(r.result, alone), f"request {r.rid}: BFS differs"
        elif r.kind == S.CC:
            alone = g.cc().cpu().numpy()
            assert np.array_equal(r.result, alone), f"request {r.rid}: CC differs"
        else:
            alone = g.pagerank(r.iters, 0.85).cpu().numpy().astype(np.float64)
            rel = np.max(np.abs(r.result.astype(np.float64) - alone) / alone)
            assert rel <= 1e-5, (r.rid, rel)
    g.status()
    return g


@pytest.mark.parametrize("realtime,rate,coalesce", [(False, 1.0, True), (True, 4000.0, True), (True, 4000.0, False)])
def test_served_queries_equal_alone(realtime, rate, coalesce):
    gp.build()
    scale, window = 14, 120_000
    stream = W.rmat_stream(scale, window + 400_000, seed=24)
    win = W.SlidingWindow(stream, window)
    V = 1 << scale
    reqs = S.make_requests(240, V, win, rate=rate, seed=9, upd_lo=10, upd_hi=4000, pr_iters=10)
    g = gp.Graph(V, leaf_size=64)
    g.update(dev(stream[:window]))
    srv = S.Server(g, max_batch_keys=1 << 14, result_slots=3, max_inflight=2, coalesce=coalesce)
    out = srv.run(reqs, realtime=realtime)
    assert all(r.done is not None and r.done >= r.arrival for r in reqs)
    assert all(r.result is not None for r in reqs if r.kind != S.UPDATE)
    n_upd = sum(r.n_keys for r in reqs if r.kind == S.UPDATE)
    assert out["edge_updates"] == n_upd
    if not realtime:
        assert out["device_batches"] < sum(r.kind == S.UPDATE for r in reqs)  # closed loop coalesces
    if not coalesce:
        assert out["device_batches"] == sum(r.kind == S.UPDATE for r in reqs)
    alone = replay_alone(V, stream[:window], reqs)
    served = np.sort(g.export_sorted().cpu().numpy().view(np.uint64))
    assert np.array_equal(served, np.sort(alone.export_sorted().cpu().numpy().view(np.uint64)))
    o = oracle.OraclePMA(V, L=64)
    o.update(stream[:window])
    for r in reqs:
        if r.kind == S.UPDATE:
            o.update(r.ins, r.dels)
    assert np.array_equal(served, np.sort(o.export_sorted()))
    assert g.check() == 0


def test_served_full_size_properties():
    """The served configuration at full size (R-MAT scale 24, 2^28 device-drawn
    samples): every query answered in the mix equals the same query on a second
    handle fed the same updates one request at a time, and the final queries (after
    the last update) satisfy what holds at any size -- BFS depths grow by at most
    one along every sampled edge, CC labels agree along sampled edges and never
    exceed the vertex id, PageRank sums to one."""
    scale = 24
    st = W.rmat_stream_device(scale, 1 << 28, seed=24)
    window = st.numel() - 5_000_000
    V = 1 << scale
    host_stream = st.cpu().numpy().view(np.uint64)
    win = W.SlidingWindow(host_stream, window)
    reqs = S.make_requests(24, V, win, rate=1.0, seed=12, upd_lo=100, upd_hi=100_000, pr_iters=10)
    t_end = reqs[-1].arrival
    final = [S.Request(len(reqs) + i, kind, t_end + 1.0 + i, src=int(host_stream[0] >> np.uint64(32)), iters=10)
             for i, kind in enumerate((S.BFS, S.CC, S.PAGERANK))]
    reqs += final
    g = gp.Graph(V, leaf_size=64)
    g.update(st[:window])
    del st
    srv = S.Server(g, max_batch_keys=1 << 20, result_slots=2, max_inflight=2)
    srv.run(reqs, realtime=False)
    alone = replay_alone(V, host_stream[:window], reqs)
    edges = g.export_sorted().cpu().numpy().view(np.uint64)
    sample = edges[np.random.default_rng(3).integers(0, edges.size, 200_000)]
    su = (sample >> np.uint64(32)).astype(np.int64)
    sv = (sample & np.uint64(0xFFFFFFFF)).astype(np.int64)
    bfs, cc, pr = (r.result for r in final)
    d = bfs.astype(np.int64)
    ok = d[su] >= 0
    assert d[final[0].src] == 0
    assert np.all(d[sv][ok] >= 0) and np.all(d[sv][ok] <= d[su][ok] + 1)
    lab = cc.view(np.uint32).astype(np.int64)
    assert np.all(lab[su] == lab[sv]) and np.all(lab <= np.arange(V))
    assert abs(float(pr.view(np.float32).astype(np.float64).sum()) - 1.0) < 1e-3
    assert g.check() == 0 and alone.check() == 0
