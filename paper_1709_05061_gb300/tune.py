"""Leaf-size autotuner for the many-graph batched update.

The leaf size L (slots per leaf segment, Sec. 3 "leaf segments") trades the
cost of the leaf pass (one warp walks L slots per touched leaf) against the
number of levels a batch climbs and the size of the count tree.  The best L
depends on the graph's size and the batch size, so each graph of a batched
workload gets its own: every candidate L is timed on a copy of the graph with a
sample batch, and the fastest is kept.  The threads per leaf segment are fixed
by the kernels (one warp per leaf in the leaf pass, one block per merged
segment), so L is the only tuned knob.
"""
from __future__ import annotations

LEAF_CANDIDATES = (32, 64, 128, 256, 512, 1024)


def pick_leaf_size(table: dict) -> int:
    """The leaf size with the smallest time in ``{L: ms}``; ties go to the smaller L."""
    if not table:
        raise ValueError("empty timing table")
    for L in table:
        if L < 2 or L > 1024 or L & (L - 1):
            raise ValueError(f"leaf size {L} is not a power of two in [2, 1024]")
    return min(sorted(table), key=lambda L: table[L])


def time_leaf_sizes(n_vertices: int, initial, ins, dels, candidates=LEAF_CANDIDATES, reps: int = 3) -> dict:
    """Median device time (ms) of one update(ins, dels) for every candidate L.

    ``initial``, ``ins`` and ``dels`` are CUDA key tensors; ``dels`` should be
    edges of ``initial`` and ``ins`` edges absent from it.  After each timed
    update the inverse update (insert ``dels``, delete ``ins``) restores the
    edge set, so every repetition times the same change."""
    import torch

    from . import Graph

    out = {}
    s = torch.cuda.current_stream()
    for L in candidates:
        g = Graph(n_vertices, leaf_size=L)
        try:
            g.update(initial)
            g.update(ins, dels)  # first use of this batch size: capture
            g.update(dels, ins)
            ts = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                g.update(ins, dels)
                e1.record(s)
                g.update(dels, ins)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            ts.sort()
            out[L] = ts[len(ts) // 2]
        finally:
            g.close()
    return out


def autotune_leaf_size(n_vertices: int, initial, ins, dels, candidates=LEAF_CANDIDATES, reps: int = 3):
    """(best L, timing table) for a graph holding ``initial`` and batches like (ins, dels)."""
    table = time_leaf_sizes(n_vertices, initial, ins, dels, candidates, reps)
    return pick_leaf_size(table), table
