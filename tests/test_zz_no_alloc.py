"""gpma_export_sorted_noalloc: the export for callers that must not allocate
device memory while they query the graph (its scratch is a fixed array inside
the library).  Its output must equal gpma_export_sorted's on two calls in a row,
which also checks that a call's leftover scratch does not disturb the next one.
This file is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1709_05061_gb300 as gp  # noqa: E402
from paper_1709_05061_gb300 import workloads as W  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def test_noalloc_export_matches_export_sorted():
    gp.build()
    V = 1 << 14
    stream = W.rmat_stream(14, 300_000, seed=21)
    g = gp.Graph(V, leaf_size=64)
    g.update(dev(stream[:250_000]), None, stats=True)
    n = g.num_edges()
    ref = torch.empty(n, dtype=torch.int64, device="cuda")
    assert gp.gpma_export_sorted(g.h, ref) == n
    for _ in range(2):
        out = torch.full((n,), -7, dtype=torch.int64, device="cuda")
        assert gp.gpma_export_sorted_noalloc(g.h, out) == n
        assert torch.equal(out, ref)
    # after a batch, both exports agree again (same array, new contents)
    g.update(dev(stream[250_000:]), dev(stream[:50_000]), stats=True)
    n2 = g.num_edges()
    ref2 = torch.empty(n2, dtype=torch.int64, device="cuda")
    assert gp.gpma_export_sorted(g.h, ref2) == n2
    out2 = torch.empty(n2, dtype=torch.int64, device="cuda")
    assert gp.gpma_export_sorted_noalloc(g.h, out2) == n2
    assert torch.equal(out2, ref2)
    # a buffer that is too small: the size needed comes back, nothing past it written
    small = torch.full((10,), -7, dtype=torch.int64, device="cuda")
    assert gp.gpma_export_sorted_noalloc(g.h, small) == -n2 - 1
    assert torch.equal(small, ref2[:10])
    g.close()


def test_noalloc_export_two_handles_same_epoch_no_allocation():
    """Two handles with the same call history (so their look-back epochs match)
    and different edges share the library's fixed scratch array: alternating
    exports must still each equal the handle's own gpma_export_sorted, which holds
    only because each call clears the words it uses.  The calls allocate nothing:
    free device memory is the same before and after each of them."""
    gp.build()
    V = 1 << 15
    sa = W.rmat_stream(15, 400_000, seed=71)
    sb = W.rmat_stream(15, 400_000, seed=72)
    ga, gb = gp.Graph(V, leaf_size=64), gp.Graph(V, leaf_size=64)
    ga.update(dev(sa), None)
    gb.update(dev(sb), None)
    na, nb = ga.num_edges(), gb.num_edges()
    refa = torch.empty(na, dtype=torch.int64, device="cuda")
    refb = torch.empty(nb, dtype=torch.int64, device="cuda")
    assert gp.gpma_export_sorted(ga.h, refa) == na
    assert gp.gpma_export_sorted(gb.h, refb) == nb
    assert not torch.equal(refa[:1000], refb[:1000])
    outa = torch.empty(na, dtype=torch.int64, device="cuda")
    outb = torch.empty(nb, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    for i in range(3):
        for g, out, n, ref in ((ga, outa, na, refa), (gb, outb, nb, refb)):
            out.fill_(-7)
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            assert gp.gpma_export_sorted_noalloc(g.h, out) == n
            free1 = torch.cuda.mem_get_info()[0]
            if i > 0:  # the first round may set up the device address of the array
                assert free1 == free0, (free0, free1)
            assert torch.equal(out, ref)
    ga.close()
    gb.close()
