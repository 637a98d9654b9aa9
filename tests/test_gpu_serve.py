"""Served stream: every query answered inside the mix (coalesced update batches,
two streams, bounded result slots) equals the oracle's answer on the same prefix
of the stream (the oracle applies the updates one request at a time): exact for
BFS and CC, within 1e-5 relative for PageRank against FP64.  The same queries run
alone on a second handle, one request at a time, give the same results as in the
mix (bit for bit).  At full size (R-MAT scale 24) the final edge set is compared
with the host's window and the final queries with the oracle's edge-list
analytics."""
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


def replay_oracle(V, initial, reqs, L=64):
    o = oracle.OraclePMA(V, L=L)
    assert o.update(initial)[0] == 0
    for r in reqs:
        if r.kind == S.UPDATE:
            assert o.update(r.ins, r.dels)[0] == 0
            continue
        if r.kind == S.BFS:
            assert np.array_equal(r.result, o.bfs(r.src)), f"request {r.rid}: BFS differs from the oracle"
        elif r.kind == S.CC:
            assert np.array_equal(r.result.view(np.uint32), o.cc()), f"request {r.rid}: CC differs from the oracle"
        else:
            ref = o.pagerank(r.iters, 0.85)
            rel = np.max(np.abs(r.result.astype(np.float64) - ref) / ref)
            assert rel <= 1e-5, (r.rid, rel)
    return o


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
    o = replay_oracle(V, stream[:window], reqs)
    alone = replay_alone(V, stream[:window], reqs)
    served = g.export_sorted().cpu().numpy().view(np.uint64)
    assert np.array_equal(served, alone.export_sorted().cpu().numpy().view(np.uint64))
    assert np.array_equal(served, o.export_sorted())  # layouts may differ: coalescing changes the batches
    assert g.check() == 0


def test_served_full_size_against_oracle():
    """The served configuration at full size (R-MAT scale 24, 2^28 device-drawn
    samples): every query answered in the mix equals the same query on a second
    handle fed the same updates one request at a time; the final edge set equals
    the host's window after the requests, edge for edge; and the final queries
    (after the last update) equal the oracle's BFS depths and CC labels on that
    edge list exactly and its FP64 PageRank within 1e-5."""
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
    assert g.check() == 0 and alone.check() == 0
    alone.close()
    # the final edge set, from the host's window (every stream edge is distinct)
    live = np.sort(win.live())
    assert np.array_equal(g.export_sorted().cpu().numpy().view(np.uint64), live)
    g.close()
    bfs, cc, pr = (r.result for r in final)
    assert np.array_equal(bfs, oracle.bfs_edges(V, live, final[0].src))
    assert np.array_equal(cc.view(np.uint32), oracle.cc_edges(V, live))
    ref = oracle.pagerank_edges(V, live, 10, 0.85)
    rel = np.max(np.abs(pr.astype(np.float64) - ref) / ref)
    assert rel <= 1e-5, rel
