"""Seeded synthetic edge streams (inputs only: no part of the update method lives here).

The paper evaluates on sliding-window streams over Reddit, Pokec, a Graph500
R-MAT graph and an Erdos-Renyi graph (Sec. 6.1, "Datasets" and "Stream
Setup"): edges arrive in timestamp order, the first part of the stream is the
initial graph, and every slide deletes the oldest edges of a fixed-size window
and inserts the newest ones.  The real datasets are not available, so every
stream here is synthetic with the shapes the paper states:

* ``er_stream``      -- uniform random directed edges (the "Random" dataset);
* ``rmat_stream``    -- R-MAT with Graph500 parameters a,b,c,d = .57,.19,.19,.05
                        (the "Graph500" dataset), vertex ids permuted by a seeded
                        permutation as the Graph500 generator does;
* ``chung_lu_stream`` -- power-law expected degrees (stand-in for Pokec).

Every stream is seeded (numpy PCG64), has no self-loops and no repeated edge:
an edge appears at most once over the whole stream, so a slide never inserts an
edge that is still inside the window.  Stream order is generation order, which
plays the role of the paper's random timestamps.  Keys are uint64
``(src << 32) | dst``.
"""
from __future__ import annotations

import numpy as np


def make_keys(src: np.ndarray, dst: np.ndarray) -> np.ndarray:
    return (src.astype(np.uint64) << np.uint64(32)) | dst.astype(np.uint64)


def split_keys(keys: np.ndarray):
    keys = np.asarray(keys, dtype=np.uint64)
    return (keys >> np.uint64(32)).astype(np.int64), (keys & np.uint64(0xFFFFFFFF)).astype(np.int64)


def _unique_in_order(keys: np.ndarray) -> np.ndarray:
    """Drop repeated keys, keeping each key's first occurrence, in stream order."""
    _, first = np.unique(keys, return_index=True)
    first.sort()
    return keys[first]


def _grow(sampler, need: int, rng, chunk: int) -> np.ndarray:
    """Draw chunks until ``need`` distinct edges exist; stream order is preserved.
    Each top-up draw is sized from the distinct-edge yield of the previous one."""
    out = np.empty(0, np.uint64)
    while out.size < need:
        cand = sampler(rng, chunk)
        before = out.size
        out = _unique_in_order(np.concatenate([out, cand]))
        gained = out.size - before
        rate = max(gained / max(chunk, 1), 1e-3)
        chunk = int(min(max((need - out.size) / rate * 1.1, 1 << 16), 1 << 27))
    return out[:need]


def er_stream(n_vertices: int, n_edges: int, seed: int = 0) -> np.ndarray:
    """``n_edges`` distinct uniform random directed edges, no self-loops."""
    def sampler(rng, n):
        s = rng.integers(0, n_vertices, n, dtype=np.int64)
        d = rng.integers(0, n_vertices, n, dtype=np.int64)
        keep = s != d
        return make_keys(s[keep], d[keep])
    rng = np.random.Generator(np.random.PCG64(seed))
    return _grow(sampler, n_edges, rng, int(n_edges * 1.1) + 16)


RMAT_GRAPH500 = (0.57, 0.19, 0.19, 0.05)


def rmat_stream(scale: int, n_edges: int, seed: int = 1, abcd=RMAT_GRAPH500,
                permute: bool = True, samples: int | None = None) -> np.ndarray:
    """R-MAT stream over 2^scale vertices.

    Each sample descends ``scale`` levels of the adjacency matrix choosing the
    quadrant (a, b, c, d) independently per level.  Vertex ids are relabelled by
    one seeded permutation (shared by src and dst).  Self-loops and repeats are
    dropped; sampling continues until ``n_edges`` distinct edges exist.
    ``samples`` fixes the size of the first draw (e.g. 2^scale * 16).
    """
    a, b, c, _ = abcd
    n = 1 << scale
    rng = np.random.Generator(np.random.PCG64(seed))
    perm = rng.permutation(n).astype(np.int64) if permute else np.arange(n, dtype=np.int64)

    def sampler(rng, m):
        src = np.zeros(m, np.int64)
        dst = np.zeros(m, np.int64)
        for _ in range(scale):
            r = rng.random(m)
            sb = r >= a + b
            db = ((r >= a) & (r < a + b)) | (r >= a + b + c)
            src = (src << 1) | sb
            dst = (dst << 1) | db
        keep = src != dst
        return make_keys(perm[src[keep]], perm[dst[keep]])
    first = samples if samples is not None else int(n_edges * 1.2) + 16
    return _grow(sampler, n_edges, rng, first)


def chung_lu_stream(n_vertices: int, n_edges: int, gamma: float = 2.1, seed: int = 7) -> np.ndarray:
    """Directed Chung-Lu stream: both endpoints drawn independently with
    probability proportional to w_i = (i+1)^(-1/(gamma-1))."""
    w = (np.arange(n_vertices, dtype=np.float64) + 1.0) ** (-1.0 / (gamma - 1.0))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]

    def sampler(rng, m):
        s = np.searchsorted(cdf, rng.random(m), side="right").clip(0, n_vertices - 1)
        d = np.searchsorted(cdf, rng.random(m), side="right").clip(0, n_vertices - 1)
        keep = s != d
        return make_keys(s[keep], d[keep])
    rng = np.random.Generator(np.random.PCG64(seed))
    return _grow(sampler, n_edges, rng, int(n_edges * 1.3) + 16)


class SlidingWindow:
    """Fixed-size window over a stream (Sec. 6.1 "Stream Setup").

    ``initial`` is the first ``window`` edges.  ``slide(k)`` returns
    (inserts, deletes): the next ``k`` stream edges and the ``k`` oldest edges
    of the window.
    """

    def __init__(self, stream: np.ndarray, window: int):
        self.stream = np.asarray(stream, dtype=np.uint64)
        self.window = int(window)
        self.head = 0               # oldest edge still in the window
        self.tail = self.window     # next edge to arrive

    @property
    def initial(self) -> np.ndarray:
        return self.stream[: self.window]

    def remaining(self) -> int:
        return self.stream.size - self.tail

    def slide(self, k: int):
        if self.tail + k > self.stream.size:
            raise IndexError("stream exhausted")
        ins = self.stream[self.tail: self.tail + k]
        dels = self.stream[self.head: self.head + k]
        self.tail += k
        self.head += k
        return ins, dels

    def live(self) -> np.ndarray:
        return self.stream[self.head: self.tail]


def log_uniform_ints(rng, lo: int, hi: int, n: int) -> np.ndarray:
    """``n`` integers whose logarithm is uniform on [log lo, log hi]."""
    return np.exp(rng.uniform(np.log(lo), np.log(hi), n)).astype(np.int64).clip(lo, hi)


class ManyGraphWorkload:
    """Independent R-MAT sliding-window streams for the batched many-graph update.

    Graph i holds a window of ``edges[i]`` edges (log-uniform in [e_lo, e_hi])
    over 2^scale[i] vertices, scale = ceil(log2(edges / 8)) clamped to [8, 22]
    (an edge factor of 8, enough distinct pairs for the stream to go on).  Every
    step gives graph i an uneven batch of ``batch[i]`` updates (log-uniform in
    [b_lo, b_hi], at most the window), half inserts and half deletes.  ``seed``
    draws the sizes; graph i's stream has seed graph_seed0 + i."""

    def __init__(self, n_graphs: int, e_lo: int, e_hi: int, b_lo: int, b_hi: int, steps: int, seed: int = 11,
                 graph_seed0: int = 1000):
        rng = np.random.Generator(np.random.PCG64(seed))
        self.edges = log_uniform_ints(rng, e_lo, e_hi, n_graphs)
        self.batch = np.minimum(log_uniform_ints(rng, b_lo, b_hi, n_graphs), self.edges) // 2 * 2
        self.batch = np.maximum(self.batch, 2)
        self.scale = np.clip(np.ceil(np.log2(self.edges / 8.0)).astype(np.int64), 8, 22)
        self.steps = int(steps)
        self.windows = []
        for i in range(n_graphs):
            half = int(self.batch[i]) // 2
            need = int(self.edges[i]) + self.steps * half
            st = rmat_stream(int(self.scale[i]), need, seed=graph_seed0 + i)
            self.windows.append(SlidingWindow(st, int(self.edges[i])))

    @property
    def n_graphs(self) -> int:
        return len(self.windows)

    def n_vertices(self, i: int) -> int:
        return 1 << int(self.scale[i])

    def slide(self):
        """(inserts, deletes) of the next step, one pair per graph."""
        return [w.slide(int(b) // 2) for w, b in zip(self.windows, self.batch)]


def rmat_stream_device(scale: int, n_samples: int, seed: int = 24, abcd=RMAT_GRAPH500):
    """R-MAT stream generated on the current CUDA device (torch's seeded Philox
    generator) for sizes where the host generator is slow: the same definition as
    ``rmat_stream`` (independent quadrant draws per level, one seeded vertex
    permutation, self-loops and repeats dropped keeping first occurrences in draw
    order), but a different random sequence.  Returns an int64 CUDA tensor of keys
    in stream order."""
    import torch
    a, b, c, _ = abcd
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    n = 1 << scale
    perm = torch.randperm(n, generator=gen, device="cuda")
    src = torch.zeros(n_samples, dtype=torch.int64, device="cuda")
    dst = torch.zeros(n_samples, dtype=torch.int64, device="cuda")
    for _ in range(scale):
        r = torch.rand(n_samples, generator=gen, device="cuda")
        sb = r >= a + b
        db = ((r >= a) & (r < a + b)) | (r >= a + b + c)
        src = (src << 1) | sb
        dst = (dst << 1) | db
        del r, sb, db
    keep = src != dst
    keys = (perm[src[keep]] << 32) | perm[dst[keep]]
    del src, dst, keep
    uniq, inv = torch.unique(keys, sorted=True, return_inverse=True)
    first = torch.full((uniq.numel(),), keys.numel(), dtype=torch.int64, device="cuda")
    first.scatter_reduce_(0, inv, torch.arange(keys.numel(), device="cuda"), reduce="amin")
    del keys, inv
    return uniq[torch.argsort(first)]
