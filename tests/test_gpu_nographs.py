"""With GPMA_NO_GRAPHS=1 every kernel of a batch is launched directly (profilers see
each launch) instead of replaying the batch's CUDA graph.  The results must not
change: a child process with graphs off applies sliding-window batches to a learned
handle (model-bucketed sort), a plain handle (radix passes) and a batched set of
handles, and every layout is compared with the oracle slot for slot."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import sys
    import numpy as np
    import torch
    sys.path.insert(0, {root!r})
    import oracle
    import paper_1709_05061_gb300 as gp
    from paper_1709_05061_gb300 import workloads as W

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()

    V = 1 << 15
    stream = W.rmat_stream(15, 600_000, seed=81)
    win = W.SlidingWindow(stream, 300_000)
    hs = [gp.Graph(V, leaf_size=64), gp.Graph(V, leaf_size=64, plain_search=True)]
    many = [gp.Graph(V, leaf_size=L) for L in (32, 64, 128)]
    o = oracle.OraclePMA(V, L=64)
    om = [oracle.OraclePMA(V, L=L) for L in (32, 64, 128)]
    for g in hs:
        g.update(dev(win.initial))
    gp.Graph.update_many(many, [dev(win.initial)] * 3, [None] * 3)
    o.update(win.initial)
    for x in om:
        x.update(win.initial)
    sorted_by_model = 0
    for b in (3000, 9000, 40_000, 120_000):
        ins, dels = win.slide(b // 2)
        st = hs[0].update(dev(ins), dev(dels), stats=True)
        sorted_by_model += st["model_sorted"]
        hs[1].update(dev(ins), dev(dels))
        gp.Graph.update_many(many, [dev(ins)] * 3, [dev(dels)] * 3)
        assert o.update(ins, dels)[0] == 0
        for x in om:
            assert x.update(ins, dels)[0] == 0
    lo = o.layout()
    for g in hs:
        g.status()
        assert np.array_equal(g.layout().cpu().numpy().view(np.uint64), lo)
        assert g.check() == 0
    for g, x in zip(many, om):
        g.status()
        assert np.array_equal(g.layout().cpu().numpy().view(np.uint64), x.layout())
    assert sorted_by_model >= 2, sorted_by_model
    print("no-graphs ok")
""")


def test_direct_launches_match_the_oracle():
    import paper_1709_05061_gb300 as gp
    gp.build()
    env = dict(os.environ, GPMA_NO_GRAPHS="1")
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "no-graphs ok" in r.stdout
