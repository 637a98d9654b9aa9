"""The update front end at the sizes where it changes form, against the oracle.

Batches of at most 4096 keys are sorted in one block.  Larger batches are sorted
by stable radix passes over tiles of 1024 keys, and their survivors and run heads
are placed from per-block counts of 256 sorted words (one a thread, below 2^19
keys) or 1024 (four a thread).  Each case checks the layout slot for slot, the batch statistics and the
exported edges, with the learned and the plain leaf search; skewed batches (one
source holding many of the batch's keys) and invalid keys in large batches too."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1709_05061_gb300 as gp  # noqa: E402
from paper_1709_05061_gb300 import workloads as W  # noqa: E402

STAT_KEYS = ("n_inserted", "n_deleted", "n_ignored", "levels_climbed", "resized", "alg_bytes", "touched_leaves",
             "covered_leaves", "merges", "delete_leaves")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.uint64)).view(np.int64)).cuda()


def host(t):
    return t.cpu().numpy().view(np.uint64)


@pytest.fixture(scope="module", autouse=True)
def built():
    gp.build()
    gp.lib()


def mixed_batch(rng, V, live, n):
    """n raw keys: new edges, inserts of stored edges, duplicates, deletes of stored
    and of absent edges, and keys on both lists."""
    k = n // 6
    new = (rng.integers(0, V, k).astype(np.uint64) << np.uint64(32)) | rng.integers(0, V, k).astype(np.uint64)
    present = live[rng.integers(0, live.size, k)] if live.size else new[:0]
    dup = new[: k // 2]
    dels = live[rng.integers(0, live.size, k)] if live.size else new[:0]
    absent = (rng.integers(0, V, k // 2).astype(np.uint64) << np.uint64(32)) | rng.integers(0, V, k // 2).astype(np.uint64)
    both = new[k // 2: k]
    ins = rng.permutation(np.concatenate([new, present, dup]))
    dl = rng.permutation(np.concatenate([dels, absent, both]))
    return ins, dl


def run_pair(V, batches, plain):
    """Apply the batches to a handle and to the oracle, comparing stats and layout
    after each; returns, per batch, whether the model-bucketed sort took it."""
    g = gp.Graph(V, leaf_size=64, plain_search=plain)
    o = oracle.OraclePMA(V, L=64)
    by_model = []
    for ins, dels in batches:
        st = g.update(dev(ins), dev(dels), stats=True)
        by_model.append(st["model_sorted"])
        rc, so = o.update(ins, dels)
        assert rc == 0
        for k in STAT_KEYS:
            assert st[k] == so[k], (k, st[k], so[k])
        lg, lo = host(g.layout()), o.layout()
        assert lg.size == lo.size and np.count_nonzero(lg != lo) == 0
    assert np.array_equal(host(g.export_sorted()), o.export_sorted())
    assert g.check() == 0
    g.close()
    return by_model


@pytest.mark.parametrize("plain", [False, True])
def test_batch_sizes_around_the_front_end_limits(plain):
    V = 1 << 16
    base = W.rmat_stream(16, 300_000, seed=61)
    rng = np.random.default_rng(61)
    batches = [(base, np.zeros(0, np.uint64))]
    live = base.copy()
    for n in (4096, 4097, 5000, 8192, 8193, 65_537, 262_145, 524_287, 524_288, 524_289):
        ins, dels = mixed_batch(rng, V, live, n)
        batches.append((ins, dels))
        live = np.array(sorted(set(live.tolist()) | set(ins.tolist()) - set(dels.tolist())), np.uint64)
    by_model = run_pair(V, batches, plain)
    # the plain handle always sorts by radix passes; the learned one buckets the
    # batches above the one-block size by model piece once they replay a graph
    assert not any(by_model) if plain else any(by_model[2:]), by_model


def test_model_bucketed_sort():
    """A learned handle with room in its root (half of its edges deleted) replays
    its graph for every batch, so the batches above the one-block size are sorted by
    bucketing on the model's pieces: layout and stats equal the oracle's at sizes
    from 4097 to 2^19 + 1 keys (with duplicates, cancellations, present inserts and
    absent deletes), for a batch crowding 20,000 new edges into one short row, whose
    bucket is too large for shared memory and is sorted in place, and for one with
    stars of 480 and 2000 new edges on other short rows (buckets near the largest one
    a warp sorts in registers, and buckets for the block sort in shared memory)."""
    V = 1 << 16
    base = W.rmat_stream(16, 1_200_000, seed=63)
    rng = np.random.default_rng(63)
    live = base[600_000:]
    batches = [(base, np.zeros(0, np.uint64)), (np.zeros(0, np.uint64), base[:600_000])]
    for n in (5462, 6000, 8193, 30_000, 65_537, 200_000, 524_289, 800_000):  # about 3n/4 keys each
        ins, dels = mixed_batch(rng, V, live, n)
        batches.append((ins, dels))
        live = np.array(sorted(set(live.tolist()) | set(ins.tolist()) - set(dels.tolist())), np.uint64)
    srcs, deg = np.unique(live >> np.uint64(32), return_counts=True)
    hub = np.uint64(srcs[np.argmin(deg)])  # a short row: it lies within one or two model pieces
    star = (hub << np.uint64(32)) | rng.permutation(V)[:20_000].astype(np.uint64)
    batches.append((star, np.zeros(0, np.uint64)))
    short = srcs[np.argsort(deg, kind="stable")[1:5]].astype(np.uint64)  # four more short rows
    stars = [(s << np.uint64(32)) | rng.permutation(V)[:c].astype(np.uint64)
             for s, c in zip(short, (480, 480, 480, 2000))]
    ins, dels = mixed_batch(rng, V, live, 8000)
    batches.append((rng.permutation(np.concatenate([ins] + stars)), dels))
    by_model = run_pair(V, batches, False)
    # every batch after the bulk load replays a graph: above the one-block size the model sorts it
    expect = [int(ins.size + dels.size > 4096) for ins, dels in batches[1:]]
    assert by_model[1:] == expect and sum(expect) >= 7, (by_model, expect)


@pytest.mark.parametrize("hot", [3000, 12_000, 20_000, 60_000])
def test_skewed_batches(hot):
    """A source with `hot` new edges in one batch of about hot + 10,000 keys: many
    equal digits in the upper radix passes, and long runs of one source."""
    V = 1 << 17
    rng = np.random.default_rng(hot)
    base = W.rmat_stream(17, 400_000, seed=62)
    hub = np.uint64(7)
    dst = rng.permutation(V)[:hot].astype(np.uint64)
    star = (hub << np.uint64(32)) | dst
    ins, dels = mixed_batch(rng, V, base, 10_000)
    ins = rng.permutation(np.concatenate([ins, star]))
    for plain in (False, True):
        by_model = run_pair(V, [(base, np.zeros(0, np.uint64)), (ins, dels), (dels, star[: hot // 2])], plain)
        if plain:
            assert not any(by_model)


def test_invalid_key_in_a_large_batch_changes_nothing():
    V = 1 << 15
    g = gp.Graph(V, leaf_size=64)
    base = W.rmat_stream(15, 200_000, seed=63)
    g.update(dev(base), None, stats=True)
    before = host(g.layout())
    rng = np.random.default_rng(63)
    ins, dels = mixed_batch(rng, V, base, 50_000)
    for bad in ([(V << 32) | 1], [(1 << 32) | V]):
        with pytest.raises(gp.GpmaError) as e:
            g.update(dev(np.concatenate([ins, np.array(bad, np.uint64)])), dev(dels), stats=True)
        assert e.value.code == gp.GPMA_EINVAL
        assert np.array_equal(host(g.layout()), before)
        g.update(dev(np.concatenate([ins, np.array(bad, np.uint64)])), dev(dels))
        with pytest.raises(gp.GpmaError):
            g.status()
        assert np.array_equal(host(g.layout()), before)
    assert g.check() == 0
    g.close()
