"""Autotuner for the many-graph batched update: leaf size and threads per leaf pass.

The leaf size L (slots per leaf segment, Sec. 3 "leaf segments") trades the
cost of the leaf pass (one warp walks L slots per touched leaf) against the
number of levels a batch climbs and the size of the count tree.  The threads
given to one segment are the other choice App. A leaves to the implementation
(its warp, block and device tiers): here one warp takes each touched leaf, and
the tuned knob is how many of those warps share a block (``leaf_warps``: 1, 2,
4 or 8), which sets the shared memory per block and so how many blocks an SM
holds.  The best pair depends on the graph's size and the batch size, so each
graph of a batched workload gets its own: every candidate is timed on a copy of
the graph with a sample batch, and the fastest is kept.  L is chosen first (at
the library's own block shape), then the warps per block at that L.
"""
from __future__ import annotations

LEAF_CANDIDATES = (32, 64, 128, 256, 512, 1024)
WARP_CANDIDATES = (1, 2, 4, 8)


def pick_leaf_size(table: dict) -> int:
    """The leaf size with the smallest time in ``{L: ms}``; ties go to the smaller L."""
    if not table:
        raise ValueError("empty timing table")
    for L in table:
        if L < 2 or L > 1024 or L & (L - 1):
            raise ValueError(f"leaf size {L} is not a power of two in [2, 1024]")
    return min(sorted(table), key=lambda L: table[L])


def pick_warps(table: dict) -> int:
    """The warps per block with the smallest time in ``{warps: ms}``; ties go to more warps."""
    if not table:
        raise ValueError("empty timing table")
    for w in table:
        if w not in WARP_CANDIDATES:
            raise ValueError(f"warps per block {w} not in {WARP_CANDIDATES}")
    return min(sorted(table, reverse=True), key=lambda w: table[w])


def time_update(n_vertices: int, initial, ins, dels, leaf_size: int, leaf_warps: int = 0, reps: int = 3) -> float:
    """Median device time (ms) of one update(ins, dels) on a graph holding ``initial``.

    ``initial``, ``ins`` and ``dels`` are CUDA key tensors; ``dels`` should be
    edges of ``initial`` and ``ins`` edges absent from it.  After each timed
    update the inverse update (insert ``dels``, delete ``ins``) restores the
    edge set, so every repetition times the same change."""
    import torch

    from . import Graph

    s = torch.cuda.current_stream()
    g = Graph(n_vertices, leaf_size=leaf_size, leaf_warps=leaf_warps)
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
        return ts[len(ts) // 2]
    finally:
        g.close()


def time_leaf_sizes(n_vertices: int, initial, ins, dels, candidates=LEAF_CANDIDATES, reps: int = 3) -> dict:
    """Median device time (ms) of one update(ins, dels) for every candidate L."""
    return {L: time_update(n_vertices, initial, ins, dels, L, 0, reps) for L in candidates}


def autotune_leaf_size(n_vertices: int, initial, ins, dels, candidates=LEAF_CANDIDATES, reps: int = 3):
    """(best L, timing table) for a graph holding ``initial`` and batches like (ins, dels)."""
    table = time_leaf_sizes(n_vertices, initial, ins, dels, candidates, reps)
    return pick_leaf_size(table), table


def autotune(n_vertices: int, initial, ins, dels, leaf_candidates=LEAF_CANDIDATES, warp_candidates=WARP_CANDIDATES,
             reps: int = 3):
    """(best L, best warps per block, {L: ms}, {warps: ms}): L first, then the
    warps per block of the one-warp-per-leaf pass at that L."""
    L, ltab = autotune_leaf_size(n_vertices, initial, ins, dels, leaf_candidates, reps)
    wtab = {w: time_update(n_vertices, initial, ins, dels, L, w, reps) for w in warp_candidates}
    return L, pick_warps(wtab), ltab, wtab
