"""Failure detection on the GPU without a GPU fault.

- Bounded waits: gpma_set_wait_limit makes every device-side wait of a handle give
  up after a few polls.  A grid barrier of gpma_bfs then runs out (its blocks
  cannot all arrive within two polls), the kernel returns, gpma_status reports
  GPMA_ETIMEOUT and the handle stays poisoned.  Export look-backs give up the
  same way; the export then says so instead of returning wrong edges.
- Allocation failures: a caller allocator that refuses the k-th request makes
  the call return GPMA_ENOMEM.  Before a batch applies anything the array stays
  unchanged, and once memory is granted again the same batch applies and matches
  the oracle; a refused root-resize array poisons the handle.  Destroy returns
  every block either way.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1709_05061_gb300 as gp  # noqa: E402
from paper_1709_05061_gb300 import workloads as W  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.uint64)).view(np.int64)).cuda()


def host(t):
    return t.cpu().numpy().view(np.uint64)


@pytest.fixture(scope="module", autouse=True)
def built():
    gp.build()
    gp.lib()


def _graph(scale, n, seed, **kw):
    V = 1 << scale
    stream = W.rmat_stream(scale, n, seed=seed)
    g = gp.Graph(V, **kw)
    g.update(dev(stream), None, stats=True)
    return g, V, stream


def test_bfs_barrier_wait_runs_out_and_poisons():
    g, V, stream = _graph(16, 400_000, seed=31)
    src = int(stream[0] >> np.uint64(32))
    ref = g.bfs(src).clone()
    assert int((ref >= 0).sum()) > 1
    gp.gpma_set_wait_limit(g.h, 1)
    g.bfs(src)  # enqueues and returns; the barrier gives up on the device
    with pytest.raises(gp.GpmaError) as e:
        g.status()
    assert e.value.code == gp.GPMA_ETIMEOUT
    # poisoned: every later call returns the same code, and nothing runs
    for call in (lambda: g.update(dev(stream[:10]), None), lambda: g.bfs(src), lambda: g.num_edges(),
                 lambda: g.status()):
        with pytest.raises(gp.GpmaError) as e:
            call()
        assert e.value.code == gp.GPMA_ETIMEOUT
    g.close()
    # the context is still usable: a new handle gives the same depths as before
    g2, _, _ = _graph(16, 400_000, seed=31)
    assert torch.equal(g2.bfs(src), ref)
    g2.close()


@pytest.mark.parametrize("noalloc", [False, True])
def test_export_wait_runs_out_and_is_reported(noalloc):
    """With a two-poll limit, some of the ~2,000 look-back tiles of the export find
    their predecessor unpublished and give up.  An export is either complete and
    right, or reports GPMA_ETIMEOUT and poisons the handle; at least one of a few
    tries must run out."""
    export = gp.gpma_export_sorted_noalloc if noalloc else gp.gpma_export_sorted
    seen = False
    for attempt in range(4):
        g, V, stream = _graph(20, 2_000_000, seed=40 + attempt)
        n = g.num_edges()
        ref = g.export_sorted()
        out = torch.empty(n, dtype=torch.int64, device="cuda")
        gp.gpma_set_wait_limit(g.h, 1)
        for _ in range(8):
            try:
                got = export(g.h, out)
            except gp.GpmaError as e:
                assert e.code == gp.GPMA_ETIMEOUT
                seen = True
                with pytest.raises(gp.GpmaError) as e2:
                    g.num_edges()
                assert e2.value.code == gp.GPMA_ETIMEOUT
                break
            assert got == n and torch.equal(out, ref)
        g.close()
        if seen:
            break
    assert seen, "no look-back wait ran out with a two-poll limit"


def test_wait_limit_zero_restores_the_default():
    g, V, stream = _graph(14, 100_000, seed=33)
    ref = g.export_sorted()
    gp.gpma_set_wait_limit(g.h, 0)
    assert torch.equal(g.export_sorted(), ref)
    g.update(dev(stream[:5000]), dev(stream[5000:10000]), stats=True)
    g.status()
    g.close()


class CountingAllocator:
    """torch's caching allocator behind gpma_allocator; once `fail_at` is set it
    refuses request number `fail_at` (counted from 1 over the allocator's life)
    and every later one."""

    def __init__(self):
        self.live = {}
        self.requests = 0
        self.fail_at = None
        self.allocator = gp.Allocator(self.alloc, self.free)

    def alloc(self, nbytes, stream):
        self.requests += 1
        if self.fail_at is not None and self.requests >= self.fail_at:
            return 0
        p = torch.cuda.caching_allocator_alloc(nbytes, stream=stream)
        self.live[p] = nbytes
        return p

    def free(self, ptr, stream):
        assert ptr in self.live
        del self.live[ptr]
        torch.cuda.caching_allocator_delete(ptr)


def _setup_counted(V, stream):
    A = CountingAllocator()
    g = gp.Graph(V, allocator=A.allocator)
    o = oracle.OraclePMA(V)
    small = stream[:2000]
    g.update(dev(small), None, stats=True)
    o.update(small)
    return A, g, o


class SizeLog(CountingAllocator):
    def __init__(self):
        super().__init__()
        self.sizes = []

    def alloc(self, nbytes, stream):
        self.sizes.append(nbytes)
        return super().alloc(nbytes, stream)


def test_allocator_failure_gives_enomem():
    """Refusals among the work-array requests of a batch (before anything is
    applied) leave the array unchanged and the handle usable; a refusal of the
    new array of a root resize (the batch's deletes and level-0 merges are then
    already applied) poisons the handle with GPMA_ENOMEM."""
    V = 1 << 14
    stream = W.rmat_stream(14, 300_000, seed=34)
    big = stream[2000:250_000]
    # where the big batch's requests go: a run with every request granted
    A = SizeLog()
    g = gp.Graph(V, allocator=A.allocator)
    g.update(dev(stream[:2000]), None, stats=True)
    first = len(A.sizes)
    st = g.update(dev(big), None, stats=True)
    assert st["resized"] == 1
    reqs = A.sizes[first:]
    C_new = g.capacity
    g.close()
    resize_at = reqs.index(8 * C_new)  # the new slot array
    assert resize_at >= 3
    for k in sorted({0, 1, resize_at // 2, resize_at - 1}):
        A, g, o = _setup_counted(V, stream)
        lay0 = g.layout().clone()
        A.fail_at = A.requests + k + 1
        with pytest.raises(gp.GpmaError) as e:
            g.update(dev(big), None, stats=True)
        assert e.value.code == gp.GPMA_ENOMEM
        assert torch.equal(g.layout(), lay0), k
        assert g.check() == 0
        # memory again: the same batch applies and matches the oracle
        A.fail_at = None
        g.update(dev(big), None, stats=True)
        o.update(big)
        assert np.array_equal(host(g.layout()), o.layout())
        assert np.array_equal(host(g.export_sorted()), o.export_sorted())
        g.close()
        assert not A.live, f"{len(A.live)} blocks not returned"
    # the resize's own array refused: poisoned, and destroy still returns everything
    A, g, o = _setup_counted(V, stream)
    A.fail_at = A.requests + resize_at + 1
    with pytest.raises(gp.GpmaError) as e:
        g.update(dev(big), None, stats=True)
    assert e.value.code == gp.GPMA_ENOMEM
    A.fail_at = None
    with pytest.raises(gp.GpmaError) as e:
        g.num_edges()
    assert e.value.code == gp.GPMA_ENOMEM
    g.close()
    assert not A.live, f"{len(A.live)} blocks not returned"


@pytest.mark.parametrize("fail_at", [1, 2, 5, 9, 14])
def test_allocator_failure_during_create(fail_at):
    A = CountingAllocator()
    A.fail_at = fail_at
    with pytest.raises(gp.GpmaError) as e:
        gp.Graph(1 << 12, allocator=A.allocator)
    assert e.value.code == gp.GPMA_ENOMEM
    torch.cuda.synchronize()
    assert not A.live, f"{len(A.live)} blocks not returned"


def test_torch_allocator_round_trip():
    V = 1 << 14
    A = gp.torch_allocator()
    before = torch.cuda.memory_allocated()
    g = gp.Graph(V, allocator=A)
    assert torch.cuda.memory_allocated() > before  # the array lives in torch's pool
    stream = W.rmat_stream(14, 200_000, seed=35)
    g.update(dev(stream[:150_000]), None)
    g.update(dev(stream[150_000:]), dev(stream[:50_000]))
    g.status()
    o = oracle.OraclePMA(V)
    o.update(stream[:150_000])
    o.update(stream[150_000:], stream[:50_000])
    assert np.array_equal(host(g.layout()), o.layout())
    assert np.array_equal(g.cc().cpu().numpy().view(np.uint32), o.cc())
    g.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before
