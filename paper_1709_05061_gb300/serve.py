"""Served graph stream: one resident GPMA+ graph answering a mixed stream of
update batches and analytic queries (the paper's framework layer, Sec. 3
"Graph Stream Buffer" / "Query Buffer" and Fig. 10's asynchronous transfers).

Requests arrive over time (host arrays for updates, a kind and a source for
queries).  The server admits them in arrival order:

* consecutive update requests that have arrived are coalesced into one device
  batch ("continuous batching") up to ``max_batch_keys`` keys, so a busy GPU
  takes fewer, larger batches;
* a query runs after every update that arrived before it and before any that
  arrived after it, so its answer is the one it would get on that prefix of the
  stream alone;
* the HBM budget bounds what is in flight: update staging buffers hold at most
  ``max_batch_keys`` keys and query results use a fixed pool of
  ``result_slots`` device buffers (a query waits for a free slot);
  ``Server.with_budget`` derives both from a byte budget.

Three CUDA streams overlap transfers with compute: host-to-device copies of
update keys and device-to-host copies of query results run on the copy stream,
updates and queries on the compute stream, ordered by events.  A PageRank query
takes its snapshot of the graph on the compute stream (in order with the
updates) and iterates on a third stream, so the updates after it need not wait
for its iterations (the snapshot holds the graph as it was).  The host keeps
at most ``max_inflight`` operations queued on the compute stream, so requests
that arrive while the GPU is busy are coalesced instead of queued one by one.

Coalescing applies several update requests as one batch.  That equals applying
them one after another when no key occurs in two of them (an insert and a
later delete of the same edge would cancel inside one batch); the sliding-window
streams used here never repeat a key, and ``coalesce=False`` turns it off.

``admit`` is the scheduling decision alone (no device code) and is what the CPU
tests exercise; ``Server`` runs the decisions on the GPU through the C ABI.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

UPDATE, BFS, CC, PAGERANK = "update", "bfs", "cc", "pagerank"


@dataclass
class Request:
    rid: int
    kind: str
    arrival: float                 # seconds from the start of the run
    ins: np.ndarray | None = None  # uint64 keys (updates)
    dels: np.ndarray | None = None
    src: int = 0                   # BFS source
    iters: int = 10                # PageRank iterations
    done: float | None = None      # completion time (seconds from the start)
    result: np.ndarray | None = None

    @property
    def n_keys(self) -> int:
        return (0 if self.ins is None else self.ins.size) + (0 if self.dels is None else self.dels.size)


@dataclass
class Op:
    kind: str                      # UPDATE or a query kind
    reqs: list = field(default_factory=list)


def admit(queue: list, head: int, now: float, max_batch_keys: int, coalesce: bool = True):
    """The next operation from ``queue[head:]`` (requests sorted by arrival), or
    None if the head request has not arrived by ``now``.  Returns (op, new_head).

    An update head takes every following update that has arrived, in order,
    while the total stays within ``max_batch_keys`` (one request always goes,
    whatever its size).  A query head goes alone."""
    if head >= len(queue) or queue[head].arrival > now:
        return None, head
    r = queue[head]
    if r.kind != UPDATE:
        return Op(r.kind, [r]), head + 1
    reqs, keys, i = [r], r.n_keys, head + 1
    while coalesce and i < len(queue):
        q = queue[i]
        if q.kind != UPDATE or q.arrival > now or keys + q.n_keys > max_batch_keys:
            break
        reqs.append(q)
        keys += q.n_keys
        i += 1
    return Op(UPDATE, reqs), i


def make_requests(n: int, n_vertices: int, window, rate: float, seed: int, upd_lo: int = 100,
                  upd_hi: int = 100_000, updates_per_query: int = 4, pr_iters: int = 10):
    """``n`` requests with Poisson arrivals at ``rate`` per second.  A request is an
    update with probability u/(u+1) (u = updates_per_query), else a query drawn
    uniformly from BFS (uniform random source), CC and PageRank.  Update sizes are
    log-uniform in [upd_lo, upd_hi], half inserts (the stream's next edges) and half
    deletes (the window's oldest), taken from ``window`` (a SlidingWindow)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, n)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for i in range(n):
        if rng.random() < updates_per_query / (updates_per_query + 1.0):
            b = int(np.exp(rng.uniform(np.log(upd_lo), np.log(upd_hi))))
            ins, dels = window.slide(max(b // 2, 1))
            out.append(Request(i, UPDATE, float(t[i]), ins=np.ascontiguousarray(ins),
                               dels=np.ascontiguousarray(dels)))
        else:
            kind = (BFS, CC, PAGERANK)[int(rng.integers(0, 3))]
            out.append(Request(i, kind, float(t[i]), src=int(rng.integers(0, n_vertices)), iters=pr_iters))
    return out


class Server:
    """Runs requests against one resident ``Graph`` with two CUDA streams."""

    def __init__(self, graph, max_batch_keys: int = 1 << 20, result_slots: int = 4, max_inflight: int = 2,
                 coalesce: bool = True, damping: float = 0.85, keep_results: bool = True):
        import torch
        self.torch = torch
        self.g = graph
        self.V = graph.n_vertices
        self.max_batch_keys = int(max_batch_keys)
        self.coalesce = coalesce
        self.damping = damping
        self.keep = keep_results
        self.max_inflight = int(max_inflight)
        self.compute = torch.cuda.Stream()
        self.copy = torch.cuda.Stream()
        self.pr_stream = torch.cuda.Stream()  # PageRank iterations over a snapshot
        self.pr_done = None                   # event: the last PageRank run has finished
        self.split_pr = True                  # snapshot + run (False once the handle refuses)
        # staging: pinned host keys and their device copies (two sets, alternating)
        self.h_keys = [torch.empty(self.max_batch_keys, dtype=torch.int64, pin_memory=True) for _ in range(2)]
        self.d_keys = [torch.empty(self.max_batch_keys, dtype=torch.int64, device="cuda") for _ in range(2)]
        self.stage_free = [None, None]     # event after which a staging set may be overwritten
        self.stage_i = 0
        self.d_res = [torch.empty(self.V, dtype=torch.int32, device="cuda") for _ in range(result_slots)]
        self.h_res = [torch.empty(self.V, dtype=torch.int32, pin_memory=True) for _ in range(result_slots)]
        self.slot_busy = [None] * result_slots  # (event, op) while a result is in flight
        self.inflight = []                      # (event, op) in completion order
        self.n_updates = 0
        self.n_batches = 0

    @staticmethod
    def budget_split(hbm_budget_bytes: int, n_vertices: int, max_slots: int = 8, max_keys: int = 1 << 22):
        """(max_batch_keys, result_slots) that fit ``hbm_budget_bytes`` of device memory:
        half of it for the two update staging buffers (8 bytes per key each), half for
        query result buffers (4 bytes per vertex each); at least one of each."""
        half = max(int(hbm_budget_bytes) // 2, 1)
        keys = max(min(half // 16, max_keys), 1024)
        slots = max(min(half // max(4 * n_vertices, 1), max_slots), 1)
        return keys, slots

    @classmethod
    def with_budget(cls, graph, hbm_budget_bytes: int, **kw):
        """A server whose staging and result buffers fit the given device-memory budget."""
        keys, slots = cls.budget_split(hbm_budget_bytes, graph.n_vertices)
        return cls(graph, max_batch_keys=keys, result_slots=slots, **kw)

    # ---- completion bookkeeping --------------------------------------------------------------
    def _poll(self, t0, block=False):
        """Retire finished operations; with ``block`` first wait for the oldest."""
        if block and self.inflight:
            self.inflight[0][0].synchronize()
        keep = []
        for ev, op, slot in self.inflight:
            if not ev.query():
                keep.append((ev, op, slot))
                continue
            now = time.perf_counter() - t0
            if slot is not None:
                r = op.reqs[0]
                if self.keep:
                    h = self.h_res[slot]
                    r.result = (h.view(self.torch.float32) if r.kind == PAGERANK else h).numpy().copy()
                self.slot_busy[slot] = None
            for r in op.reqs:
                r.done = now
        self.inflight = keep

    # ---- issuing ------------------------------------------------------------------------------
    def _issue_update(self, op):
        torch = self.torch
        ins = np.concatenate([r.ins for r in op.reqs if r.ins is not None and r.ins.size] or [np.empty(0, np.uint64)])
        dels = np.concatenate([r.dels for r in op.reqs if r.dels is not None and r.dels.size] or
                              [np.empty(0, np.uint64)])
        ni, nd = ins.size, dels.size
        i = self.stage_i
        self.stage_i ^= 1
        if self.stage_free[i] is not None:
            self.stage_free[i].synchronize()  # the copy that last used this set is done
        hk = self.h_keys[i].numpy().view(np.uint64)
        hk[:ni] = ins
        hk[ni:ni + nd] = dels
        dk = self.d_keys[i]
        with torch.cuda.stream(self.copy):
            dk[: ni + nd].copy_(self.h_keys[i][: ni + nd], non_blocking=True)
            copied = torch.cuda.Event()
            copied.record(self.copy)
        self.compute.wait_event(copied)
        self.g.update(dk[:ni] if ni else None, dk[ni:ni + nd] if nd else None, stream=self.compute)
        done = torch.cuda.Event()
        done.record(self.compute)
        self.stage_free[i] = done
        self.inflight.append((done, op, None))
        self.n_updates += ni + nd
        self.n_batches += 1

    def _issue_query(self, op, t0):
        torch = self.torch
        from . import gpma_bfs, gpma_cc, gpma_pagerank, gpma_pagerank_run, gpma_pagerank_snapshot
        while True:
            free = [k for k, b in enumerate(self.slot_busy) if b is None]
            if free:
                break
            self._poll(t0, block=True)
        k = free[0]
        r = op.reqs[0]
        out = self.d_res[k]
        ran = torch.cuda.Event()
        if r.kind == BFS:
            gpma_bfs(self.g.h, r.src, out, self.compute)
            ran.record(self.compute)
        elif r.kind == CC:
            gpma_cc(self.g.h, out, self.compute)
            ran.record(self.compute)
        else:
            if self.pr_done is not None:
                self.compute.wait_event(self.pr_done)  # the snapshot buffers are free again
            if self.split_pr and gpma_pagerank_snapshot(self.g.h, self.compute):
                snap = torch.cuda.Event()
                snap.record(self.compute)
                self.pr_stream.wait_event(snap)
                gpma_pagerank_run(self.g.h, r.iters, self.damping, out.view(torch.float32), self.pr_stream)
                ran.record(self.pr_stream)
                self.pr_done = ran
            else:
                self.split_pr = False
                gpma_pagerank(self.g.h, r.iters, self.damping, out.view(torch.float32), self.compute)
                ran.record(self.compute)
        self.copy.wait_event(ran)
        with torch.cuda.stream(self.copy):
            self.h_res[k].copy_(out, non_blocking=True)
            back = torch.cuda.Event()
            back.record(self.copy)
        self.slot_busy[k] = op
        self.inflight.append((back, op, k))

    def run(self, requests: list, realtime: bool = True):
        """Serve ``requests`` (sorted by arrival).  With ``realtime`` the host waits
        for each arrival time; without it every request counts as arrived at once
        (closed loop, for capacity; their arrival times are then set to 0, so the
        latencies are measured from the start).  Returns a summary dict."""
        torch = self.torch
        if not realtime:
            for r in requests:
                r.arrival = 0.0
        self.n_updates = self.n_batches = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        head = 0
        while head < len(requests) or self.inflight:
            self._poll(t0)
            if head < len(requests) and len(self.inflight) < self.max_inflight:
                now = time.perf_counter() - t0 if realtime else float("inf")
                op, head = admit(requests, head, now, self.max_batch_keys, self.coalesce)
                if op is None:
                    continue  # the next request has not arrived: spin
                if op.kind == UPDATE:
                    self._issue_update(op)
                else:
                    self._issue_query(op, t0)
            elif self.inflight:
                self._poll(t0, block=True)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        self.g.status(self.compute)
        return summarize(requests, wall, self.n_updates, self.n_batches)


def summarize(requests: list, wall: float, n_updates: int, n_batches: int) -> dict:
    lat = {k: [] for k in (UPDATE, BFS, CC, PAGERANK)}
    for r in requests:
        lat[r.kind].append((r.done - r.arrival) * 1e3)
    allq = lat[BFS] + lat[CC] + lat[PAGERANK]
    every = lat[UPDATE] + allq

    def pct(v, p):
        return float(np.percentile(v, p)) if v else None
    return {"requests": len(requests), "wall_s": wall, "edge_updates": n_updates, "device_batches": n_batches,
            "edge_updates_per_s": n_updates / wall if wall > 0 else None,
            "requests_per_s": len(requests) / wall if wall > 0 else None,
            "p50_ms": pct(every, 50), "p99_ms": pct(every, 99),
            "update_p50_ms": pct(lat[UPDATE], 50), "update_p99_ms": pct(lat[UPDATE], 99),
            "query_p50_ms": pct(allq, 50), "query_p99_ms": pct(allq, 99),
            "per_kind_p50_ms": {k: pct(v, 50) for k, v in lat.items()}}
