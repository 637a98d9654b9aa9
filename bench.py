#!/usr/bin/env python3
"""Benchmark of the GPMA+ hot path on GB300 (one JSON line on stdout).

Workload: R-MAT scale 20 (2^20 vertices, a,b,c,d = .57/.19/.19/.05, seeded
vertex permutation, no self-loops, no repeated edge), a sliding window of
16,000,000 edges kept in one GPMA+ array (leaf size 64), and one step =
  one update batch (B/2 newest stream edges inserted, B/2 oldest deleted)
  + PageRank (20 iterations, d = 0.85) + BFS from a seeded source + weakly
  connected components,
all through the libgpma C ABI.  `value` is edge updates per second over whole
steps; the batch-size sweep reports update-only throughput, p50/p99 latency and
the fraction of HBM bandwidth against algorithmic bytes, beside a full
sort-and-rebuild CSR baseline on the same GPU (torch sort, library code).

--impl reference times the CPU oracle (tests' reference implementation) on the
same steps on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
# more hardware work queues: queries run on their own streams, and the batches of the
# many-graph update that may resize their array run on one side stream each
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
sys.path.insert(0, ROOT)

SCALE, WINDOW, LEAF = 20, 16_000_000, 64
SWEEP = (100, 1000, 10_000, 100_000, 1_000_000)
SWEEP_WARM, SWEEP_TIMED = 3, 10
PR_ITERS, DAMPING = 20, 0.85
# steps run again after the timed region with per-phase events on (phase times,
# the dominant kernel's per-launch time); the timed region itself records none
PROFILED_STEPS = 10
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the PageRank sum
# pass on the default workload (R-MAT scale 20, 16M-edge window, 2^25 slots), from one ncu
# capture of each kernel as it stands (profiles/): push pass 285,246,720 read + 3,048,448
# written; bucketed iteration (8192-head buckets, 2 blocks of 1024 threads a bucket)
# 136,487,424 read + 3,047,680 written
PR_PASS_TRAFFIC = {"k_pr_scatter": 288_295_168, "k_pb_iter": 139_535_104}
# the library buckets the edges for PageRank on graphs of at most 2^25 vertices
PB_MAX_V = 1 << 25
METRIC = "edge updates/sec vs batch size (+HBM GB/s frac); p50/p99 update+query latency"
L2_BYTES = 129 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpma", choices=["gpma", "reference"])
    ap.add_argument("--batch", type=int, default=1_000_000)
    ap.add_argument("--scale", type=int, default=SCALE)
    ap.add_argument("--window", type=int, default=WINDOW)
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-studies", action="store_true",
                    help="skip the scale-24 update sweep and served stream, the learned-search and the "
                         "many-graph studies that the default run adds to the line")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--push-pagerank", action="store_true",
                    help="PageRank by the push pass (one L2 reduction per edge) instead of the bucketed pass")
    ap.add_argument("--learned-study", action="store_true",
                    help="only compare the learned and the plain leaf search on the power-law workload")
    ap.add_argument("--serve-study", action="store_true",
                    help="only run the served stream (R-MAT scale 24, Poisson updates and queries)")
    ap.add_argument("--serve-requests", type=int, default=1500)
    ap.add_argument("--many-study", action="store_true",
                    help="only time the batched many-graph update (64 uneven R-MAT graphs)")
    ap.add_argument("--profile-case", choices=["pr", "update", "bfs", "cc"],
                    help="load the window, run one call of this kind --repeat times and exit (a small, "
                         "self-contained run for ncu; GPMA_NO_GRAPHS=1 launches an update's kernels directly)")
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--plain-search", action="store_true", help="profile case: binary leaf search only")
    ap.add_argument("--graph", choices=["rmat", "chunglu"], default="rmat",
                    help="profile case: R-MAT window, or the power-law graph of the learned-search study "
                         "(1.6M vertices, 30M edges; batches of --batch keys, 70%% new edges, 30%% random live edges)")
    return ap.parse_args()


def workload_config(a, world):
    return {
        "workload": f"rmat-s{a.scale}-window{a.window}-batch{a.batch}",
        "graph": f"R-MAT scale {a.scale}, a,b,c,d=.57/.19/.19/.05, seeded permutation, no self-loops/repeats",
        "n_vertices": 1 << a.scale,
        "window_edges": a.window,
        "batch": a.batch,
        "batch_mix": "B/2 newest stream edges inserted + B/2 oldest window edges deleted",
        "step": f"update batch + PageRank({PR_ITERS}, d={DAMPING}) + BFS(seeded source) + weakly connected components",
        "leaf_size": LEAF,
        "l2": "inputs larger than L2: 268 MB array streamed by every step; sweep flushes L2 between batches",
        "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
        "streams": "update + PageRank on one stream, BFS + CC on a second",
    }


def stream_needed(a, reference: bool):
    half = a.batch // 2
    n = a.window + half * (a.warmup + a.steps)
    if reference:
        return n
    n += half * PROFILED_STEPS
    if not a.no_e2e:
        n += half * (a.warmup + a.steps)
    if not a.no_sweep:
        n += sum((SWEEP_WARM + SWEEP_TIMED) * (b // 2) for b in SWEEP)
    return n


def max_over_ranks(x: float, dist, device) -> float:
    """The largest ``x`` over all ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, batch: int, steps: int, ms: float) -> float:
    """Whole-job edge updates per second: every rank applies ``steps`` batches of
    ``batch`` updates to its own replica; ``ms`` is the max over ranks."""
    return world * batch * steps / (ms * 1e-3)


def make_stream(a, rank, reference=False):
    from paper_1709_05061_gb300 import workloads as W
    return W.rmat_stream(a.scale, stream_needed(a, reference), seed=a.seed + 1000 * rank,
                         samples=(1 << a.scale) * 16)


def bfs_source(stream):
    return int(stream[0] >> np.uint64(32))


# ---- clocks during the timed region ------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None
        self.lines = []

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "20"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t_end = time.perf_counter() + 5.0  # the sampler is running before the timed region starts
            while not self.lines and time.perf_counter() < t_end:
                time.sleep(0.005)
        except Exception:
            self.p = None
        self.t0 = time.perf_counter()
        return self

    def _read(self):
        for line in self.p.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def __exit__(self, *exc):
        self.t1 = time.perf_counter()
        if self.p:
            time.sleep(0.025)  # one more sample after the region
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        # samples taken inside the region, and the first one after it
        inside = [ln for t, ln in self.lines if self.t0 <= t <= self.t1]
        after = [ln for t, ln in self.lines if t > self.t1][:1]
        for ln in inside + after:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def hold_gpu(cycles: int = 200_000):
    """Keep the GPU busy for ~0.1 ms so that the host has enqueued the next call's
    launches before the device reaches them: the call's events then measure device
    time, not the host's enqueue latency (which the first call after host work pays)."""
    import torch
    torch.cuda._sleep(cycles)


def alg_bytes_table(st: dict, n_raw: int, C_old: int, C_new: int) -> int:
    """Algorithmic bytes of one batch by the measurement plan's formula: 16 B per
    raw update key (read once, written once while staging), a 512-byte read of
    every leaf holding a delete, an 8-byte EMPTY store per delete, a read and a
    write of every slot of the merged segments, and on a resize a read of the
    old array and a write of the new one."""
    a = 16 * n_raw + 8 * LEAF * st["delete_leaves"] + 8 * st["n_deleted"] + 16 * LEAF * st["covered_leaves"]
    if st["resized"]:
        a += 8 * C_old + 8 * C_new
    return a


def measured_hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def sweep_entry(b, times, algb, algt, peak):
    """p50/p99 of the per-batch device times, and the HBM fraction by the library's
    algorithmic bytes (alg_*) and by the measurement plan's formula (table_*)."""
    med = statistics.median(times)
    gbs = statistics.median([x / (t * 1e-3) / 1e9 for x, t in zip(algb, times)])
    gbt = statistics.median([x / (t * 1e-3) / 1e9 for x, t in zip(algt, times)])
    return {"batch": b, "updates_per_s": b / (med * 1e-3), "p50_ms": med,
            "p99_ms": float(np.percentile(times, 99)),
            "alg_bytes": int(statistics.median(algb)), "alg_GBps": gbs, "hbm_frac": gbs / peak,
            "table_alg_bytes": int(statistics.median(algt)), "table_GBps": gbt, "table_hbm_frac": gbt / peak}


# ---- the GPU arm -----------------------------------------------------------------------------------
def run_gpu(a, stream, rank, world, dist):
    import torch
    import paper_1709_05061_gb300 as gp
    from paper_1709_05061_gb300 import workloads as W

    gp.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    V = 1 << a.scale
    win = W.SlidingWindow(stream, a.window)
    half = a.batch // 2

    def to_dev(x):
        return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).to(dev)

    g = gp.Graph(V, leaf_size=LEAF, push_pagerank=a.push_pagerank)
    st = g.update(to_dev(win.initial), None, stats=True)
    torch.cuda.synchronize()
    src = bfs_source(stream)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)
    out = {}

    # -- batch-size sweep: update-only device time, algorithmic bytes, rebuild baseline ----------
    peak, peak_kind = measured_hbm_peak()
    if not a.no_sweep and rank == 0:
        live = to_dev(np.sort(win.live()))
        sweep = []
        for b in SWEEP:
            times, algb, algt, rb_times = [], [], [], []
            for it in range(SWEEP_WARM + SWEEP_TIMED):
                ins, dels = win.slide(b // 2)
                di, dd = to_dev(ins), to_dev(dels)
                flush.zero_()
                c_old = g.capacity
                hold_gpu()
                gp.gpma_profile_enable(g.h, True)
                s = g.update(di, dd, stats=True)
                p = gp.gpma_profile_read(g.h, reset=True)
                gp.gpma_profile_enable(g.h, False)
                ms = p["update"]["ms"]
                # sort-and-rebuild CSR baseline on the same batch
                flush.zero_()
                hold_gpu()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                keep = ~torch.isin(live, dd)
                merged = torch.cat([live[keep], di])
                live2, _ = torch.sort(merged)
                rowptr = torch.searchsorted(live2 >> 32, torch.arange(V + 1, device=dev, dtype=torch.int64))
                e1.record()
                torch.cuda.synchronize()
                live = live2
                del rowptr
                if it >= SWEEP_WARM:
                    times.append(ms)
                    algb.append(s["alg_bytes"])
                    algt.append(alg_bytes_table(s, b, c_old, g.capacity))
                    rb_times.append(e0.elapsed_time(e1))
            sweep.append(sweep_entry(b, times, algb, algt, peak))
            sweep[-1]["rebuild_p50_ms"] = statistics.median(rb_times)
            sweep[-1]["speedup_vs_rebuild"] = statistics.median(rb_times) / sweep[-1]["p50_ms"]
        out["sweep"] = sweep
        del live
    # the sweep slid only rank 0's window; every rank now continues from its own state

    ins_all, del_all = [], []
    for _ in range(a.warmup + a.steps + PROFILED_STEPS):
        ins, dels = win.slide(half)
        ins_all.append(to_dev(ins))
        del_all.append(to_dev(dels))
    rank_t = torch.empty(V, dtype=torch.float32, device=dev)
    depth = torch.empty(V, dtype=torch.int32, device=dev)
    label = torch.empty(V, dtype=torch.int32, device=dev)

    # The three queries only read the array: BFS and CC run on a second stream beside
    # PageRank, and the next update waits for both.  That stream has the higher priority:
    # BFS and CC finish sooner and the PageRank iterations then run alone (measured 1%
    # faster per step; the opposite priority measured 3% slower)
    cs, qs = torch.cuda.current_stream(), torch.cuda.Stream(priority=-1)
    ev_upd, ev_q = torch.cuda.Event(), torch.cuda.Event()

    def queries(rank_o, depth_o, label_o):
        ev_upd.record(cs)
        qs.wait_event(ev_upd)
        gp.gpma_bfs(g.h, src, depth_o, stream=qs)
        gp.gpma_cc(g.h, label_o, stream=qs)
        gp.gpma_pagerank(g.h, PR_ITERS, DAMPING, rank_o)
        ev_q.record(qs)
        cs.wait_event(ev_q)

    def step(i):
        gp.gpma_update_batch(g.h, ins_all[i], del_all[i])
        queries(rank_t, depth, label)

    # first calls on one stream: they allocate the queries' buffers
    gp.gpma_pagerank(g.h, PR_ITERS, DAMPING, rank_t)
    gp.gpma_bfs(g.h, src, depth)
    gp.gpma_cc(g.h, label)
    torch.cuda.synchronize()

    for i in range(a.warmup):
        step(i)
    gp.gpma_status(g.h)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = gp.gpma_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        e0.record()
        for i in range(a.warmup, a.warmup + a.steps):
            step(i)
        e1.record()
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches = gp.gpma_launch_count() - l0
    gp.gpma_status(g.h)
    # the same steps again with an event pair around every phase and PageRank launch
    # (the timed region above records none): phase times and per-launch kernel times
    gp.gpma_profile_read(g.h, reset=True)
    gp.gpma_profile_enable(g.h, True)
    p0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0[0].record()
    for i in range(a.warmup + a.steps, a.warmup + a.steps + PROFILED_STEPS):
        step(i)
    p0[1].record()
    torch.cuda.synchronize()
    gp.gpma_profile_enable(g.h, False)
    prof = gp.gpma_profile_read(g.h, reset=True)
    gp.gpma_status(g.h)
    out["profiled_ms_per_step"] = p0[0].elapsed_time(p0[1]) / PROFILED_STEPS
    ms = e0.elapsed_time(e1)
    ms = max_over_ranks(ms, dist, dev)
    out["ms_total"] = ms
    out["launches"] = launches
    out["profile"] = prof
    out["clocks"] = clk.summary()
    out["capacity"] = g.capacity
    out["n_edges"] = g.num_edges()
    C, Vn = g.capacity, V
    # dominant kernel by device time inside the timed region
    pr = prof["pr_scatter"]
    per_launch_ms = pr["ms"] / max(pr["count"], 1)
    if a.push_pagerank or Vn > PB_MAX_V:
        kname, what = "k_pr_scatter", "PageRank push pass over the gapped array"
        alg_pr = 8 * C + 20 * Vn  # stream every slot; read contrib, read+write the fixed-point sum once per vertex
    else:
        kname, what = "k_pb_iter", "PageRank iteration over the head-bucketed edge copy, update fused"
        # read every edge of the copy once; per vertex read its contribution and out-degree
        # once and write the next contribution
        alg_pr = 8 * out["n_edges"] + 12 * Vn
    out["roofline"] = {
        "kernel": f"{kname} ({what})",
        "bound": "hbm", "achieved": alg_pr / (per_launch_ms * 1e-3) / 1e9, "peak": peak,
        "peak_kind": peak_kind, "unit": "GB/s",
        "frac": alg_pr / (per_launch_ms * 1e-3) / 1e9 / peak,
        "traffic": PR_PASS_TRAFFIC[kname] if (a.scale, a.window) == (SCALE, WINDOW) else None,
        "alg_bytes_per_launch": alg_pr, "launch_ms": per_launch_ms,
        "share_of_step": pr["ms"] / (out["profiled_ms_per_step"] * PROFILED_STEPS),
        "timing": f"per-launch CUDA events on the launching stream over {PROFILED_STEPS} steps run right "
                  f"after the timed region (the timed region itself records no events)",
    }
    if prof["pr_bucket"]["count"]:
        out["roofline"]["bucketing_ms_per_call"] = prof["pr_bucket"]["ms"] / prof["pr_bucket"]["count"]
    # the queries in edge terms: stored edges times PageRank iterations per second of the
    # PageRank call, and stored edges per second of one BFS / CC call (device time of the
    # calls inside the timed region, where BFS and CC overlap PageRank)
    per_call = {k: prof[k]["ms"] / max(prof[k]["count"], 1) for k in ("pagerank", "bfs", "cc")}
    out["analytics"] = {
        "pagerank_ms": per_call["pagerank"], "bfs_ms": per_call["bfs"], "cc_ms": per_call["cc"],
        "pagerank_edge_iters_per_s": out["n_edges"] * PR_ITERS / (per_call["pagerank"] * 1e-3)
        if per_call["pagerank"] else None,
        "bfs_edges_per_s": out["n_edges"] / (per_call["bfs"] * 1e-3) if per_call["bfs"] else None,
        "cc_edges_per_s": out["n_edges"] / (per_call["cc"] * 1e-3) if per_call["cc"] else None,
    }
    # Inside the step BFS and CC share the GPU with PageRank, which stretches its launches;
    # the same kernel timed once more after the timed region with the GPU to itself:
    torch.cuda.synchronize()
    gp.gpma_profile_read(g.h, reset=True)
    gp.gpma_profile_enable(g.h, True)
    gp.gpma_pagerank(g.h, PR_ITERS, DAMPING, rank_t)
    torch.cuda.synchronize()
    gp.gpma_profile_enable(g.h, False)
    alone = gp.gpma_profile_read(g.h, reset=True)
    alone_ms = alone["pr_scatter"]["ms"] / max(alone["pr_scatter"]["count"], 1)
    out["roofline"]["alone"] = {"launch_ms": alone_ms, "achieved": alg_pr / (alone_ms * 1e-3) / 1e9,
                                "frac": alg_pr / (alone_ms * 1e-3) / 1e9 / peak}

    # -- e2e: host (pinned) inputs copied in and results copied out every step ---------------------
    if not a.no_e2e:
        h_ins, h_del = [], []
        for _ in range(a.warmup + a.steps):
            ins, dels = win.slide(half)
            h_ins.append(torch.from_numpy(np.ascontiguousarray(ins).view(np.int64)).pin_memory())
            h_del.append(torch.from_numpy(np.ascontiguousarray(dels).view(np.int64)).pin_memory())
        # Two sets of device inputs and host outputs: while step i computes on the default
        # stream, a copy stream brings in step i+1's inputs; step i's results go back while
        # step i+1 computes, and the host waits for them before it moves on.
        d_ins = [torch.empty(half, dtype=torch.int64, device=dev) for _ in range(2)]
        d_del = [torch.empty(half, dtype=torch.int64, device=dev) for _ in range(2)]
        d_rank = [rank_t, torch.empty_like(rank_t)]
        d_depth = [depth, torch.empty_like(depth)]
        d_label = [label, torch.empty_like(label)]
        o_rank = [torch.empty(V, dtype=torch.float32).pin_memory() for _ in range(2)]
        o_depth = [torch.empty(V, dtype=torch.int32).pin_memory() for _ in range(2)]
        o_label = [torch.empty(V, dtype=torch.int32).pin_memory() for _ in range(2)]
        cs, xs = torch.cuda.current_stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_done = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]

        def fetch(i):  # inputs of step i into set i % 2, once step i - 2 is done with it
            b = i % 2
            with torch.cuda.stream(xs):
                if i >= 2:
                    xs.wait_event(ev_done[b])
                d_ins[b].copy_(h_ins[i], non_blocking=True)
                d_del[b].copy_(h_del[i], non_blocking=True)
                ev_in[b].record(xs)

        def run(i, last):
            b = i % 2
            cs.wait_event(ev_in[b])
            if i >= 2:
                cs.wait_event(ev_out[b])  # step i-2's results have left set b
            gp.gpma_update_batch(g.h, d_ins[b], d_del[b])
            queries(d_rank[b], d_depth[b], d_label[b])
            ev_done[b].record(cs)
            if not last:
                fetch(i + 1)
            with torch.cuda.stream(xs):
                xs.wait_event(ev_done[b])
                o_rank[b].copy_(d_rank[b], non_blocking=True)
                o_depth[b].copy_(d_depth[b], non_blocking=True)
                o_label[b].copy_(d_label[b], non_blocking=True)
                ev_out[b].record(xs)

        def steps(first, n):
            fetch(first)
            for i in range(first, first + n):
                run(i, i == first + n - 1)
                if i > first:
                    ev_out[(i - 1) % 2].synchronize()  # the host has step i-1's results
            ev_out[(first + n - 1) % 2].synchronize()

        steps(0, a.warmup)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record()
        steps(a.warmup, a.steps)
        f1.record()
        torch.cuda.synchronize()
        wall = (time.perf_counter() - t0) * 1e3
        ems = max(f0.elapsed_time(f1), wall)
        ems = max_over_ranks(ems, dist, dev)
        out["e2e"] = {"value": job_value(world, a.batch, a.steps, ems), "unit": "edge updates/s",
                      "h2d_bytes_per_step": 2 * half * 8, "d2h_bytes_per_step": 3 * 4 * V,
                      "ms_per_step": ems / a.steps}
        gp.gpma_status(g.h)
    g.close()
    return out


# ---- learned vs plain leaf search (power-law workload) -----------------------------------------------
def learned_study(a):
    """Chung-Lu graph (1.6M vertices, 30M edges, degree exponent 2.1, seed 7),
    batches of 1e5 updates: 70% new edges inserted, 30% random live edges deleted.
    The same batches go to a handle with the learned leaf search and one with
    plain binary search; per-batch device time from the library's events, and the
    two arrays compared slot for slot at the end."""
    import torch
    import paper_1709_05061_gb300 as gp
    from paper_1709_05061_gb300 import workloads as W
    gp.build()
    torch.cuda.set_device(0)
    V, E0, B = 1_600_000, 30_000_000, 100_000
    n_ins, n_del = int(B * 0.7), B - int(B * 0.7)
    warm, timed = 3, 10
    stream = W.chung_lu_stream(V, E0 + (warm + timed) * n_ins, gamma=2.1, seed=7)
    rng = np.random.default_rng(7)
    live = stream[:E0].copy()

    def dev(x):
        return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda()
    graphs = {"learned": gp.Graph(V, leaf_size=LEAF), "plain": gp.Graph(V, leaf_size=LEAF, plain_search=True)}
    for g in graphs.values():
        g.update(dev(stream[:E0]), None, stats=True)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")
    times = {k: [] for k in graphs}
    clk = ClockSampler(torch.cuda.current_device()).__enter__()
    for i in range(warm + timed):
        ins = stream[E0 + i * n_ins: E0 + (i + 1) * n_ins]
        pick = rng.choice(live.size, n_del, replace=False)
        dels = live[pick]
        keep = np.ones(live.size, bool)
        keep[pick] = False
        live = np.concatenate([live[keep], ins])
        di, dd = dev(ins), dev(dels)
        # alternate which handle goes first, and let the host run ahead of the device
        for name in (("learned", "plain") if i % 2 == 0 else ("plain", "learned")):
            g = graphs[name]
            flush.zero_()
            hold_gpu()
            gp.gpma_profile_enable(g.h, True)
            g.update(di, dd, stats=True)
            p = gp.gpma_profile_read(g.h, reset=True)
            gp.gpma_profile_enable(g.h, False)
            if i >= warm:
                times[name].append(p["update"]["ms"])
    clk.__exit__(None, None, None)
    same = bool(torch.equal(graphs["learned"].layout(), graphs["plain"].layout()))
    out = {"workload": f"chung-lu V={V} E={E0} gamma=2.1 seed=7, batch {B} (70% insert / 30% random delete)",
           "clocks": clk.summary(),
           "plain_p50_ms": statistics.median(times["plain"]), "learned_p50_ms": statistics.median(times["learned"]),
           "layouts_identical": same, "capacity_slots": graphs["plain"].capacity,
           "plain_ms": times["plain"], "learned_ms": times["learned"]}
    out["speedup"] = out["plain_p50_ms"] / out["learned_p50_ms"]
    for g in graphs.values():
        g.close()
    return out


def many_study(a):
    """64 independent R-MAT graphs, window sizes log-uniform in [2^10, 2^22]
    edges, per-step batches log-uniform in [64, 2^18] updates (half inserts, half
    deletes).  Per step: all 64 batches through gpma_update_many (one CUDA graph
    whose every stage is one launch over all graphs' work) against the same
    batches applied one graph after another on one stream, at leaf size 64 and at
    the leaf size and warps per leaf-pass block the autotuner picks per graph.
    Batches are resident on the device before timing; device time with CUDA events
    on the calling stream; the batched and the sequential arrays are compared slot
    for slot at the end."""
    import torch
    import paper_1709_05061_gb300 as gp
    from paper_1709_05061_gb300 import tune
    from paper_1709_05061_gb300 import workloads as W
    gp.build()
    torch.cuda.set_device(0)
    warm, timed = 3, 10
    wl = W.ManyGraphWorkload(64, 1 << 10, 1 << 22, 64, 1 << 18, steps=warm + timed, seed=11)
    n = wl.n_graphs

    def dev(x):
        return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda()
    init = [dev(w.initial) for w in wl.windows]
    batches = [[(dev(i), dev(d)) for i, d in wl.slide()] for _ in range(warm + timed)]
    # autotune on the first step's batches, on copies of the initial graphs
    t0 = time.perf_counter()
    tuned, warps = [], []
    for i in range(n):
        L, w, _, _ = tune.autotune(wl.n_vertices(i), init[i], batches[0][i][0], batches[0][i][1], reps=3)
        tuned.append(L)
        warps.append(w)
    tune_s = time.perf_counter() - t0
    s = torch.cuda.current_stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")
    res = {}
    layouts = {}
    clk = ClockSampler(torch.cuda.current_device()).__enter__()
    for label, sizes, wpb in (("L64", [64] * n, [0] * n), ("tuned", tuned, warps)):
        for mode in ("sequential", "batched"):
            gs = [gp.Graph(wl.n_vertices(i), leaf_size=sizes[i], leaf_warps=wpb[i]) for i in range(n)]
            gp.Graph.update_many(gs, init, [None] * n)
            ts = []
            for k, b in enumerate(batches):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                if mode == "batched":
                    gp.Graph.update_many(gs, [x[0] for x in b], [x[1] for x in b])
                else:
                    for g, (bi, bd) in zip(gs, b):
                        g.update(bi, bd)
                e1.record(s)
                e1.synchronize()
                if k >= warm:
                    ts.append(e0.elapsed_time(e1))
            for g in gs:
                g.status()
            layouts[(label, mode)] = [g.layout().cpu() for g in gs]
            for g in gs:
                g.close()
            ms = statistics.median(ts)
            res[f"{label}_{mode}"] = {"p50_ms": ms, "p99_ms": float(np.percentile(ts, 99)),
                                     "edge_updates_per_s": float(wl.batch.sum()) / (ms * 1e-3)}
        same = all(torch.equal(x, y) for x, y in zip(layouts[(label, "sequential")], layouts[(label, "batched")]))
        res[f"{label}_batched_equals_sequential"] = same
    clk.__exit__(None, None, None)
    res["clocks"] = clk.summary()
    res["workload"] = (f"64 R-MAT graphs (.57/.19/.19/.05), windows log-uniform in [2^10, 2^22] edges "
                       f"(total {int(wl.edges.sum())}), batches log-uniform in [64, 2^18] "
                       f"(total {int(wl.batch.sum())} updates per step), size seed 11, graph seeds 1000+g")
    res["tuned_leaf_sizes"] = {str(L): tuned.count(L) for L in sorted(set(tuned))}
    res["tuned_leaf_warps"] = {str(w): warps.count(w) for w in sorted(set(warps))}
    res["autotune_seconds"] = tune_s
    res["speedup_batched_vs_sequential_L64"] = res["L64_sequential"]["p50_ms"] / res["L64_batched"]["p50_ms"]
    res["speedup_tuned_batched_vs_L64_sequential"] = res["L64_sequential"]["p50_ms"] / res["tuned_batched"]["p50_ms"]
    return res


def serve_study(a):
    """Served stream on a resident R-MAT scale-24 graph (2^28 samples, seed 24,
    generated on the device; about 2.6e8 distinct edges, the last 7e7 of the
    stream held back as future inserts).  Requests: Poisson arrivals, updates of
    log-uniform 1e2..1e5 keys (half new edges, half the window's oldest) mixed 4:1
    with queries (BFS from a uniform random source, CC, PageRank-10), update keys
    arriving in pinned host memory.  First a closed loop measures capacity
    (requests/s with every request available at once), then open loops at 50%,
    80% and 95% of it report p50/p99 latency (arrival to result on the host) and
    sustained edge updates/s."""
    import torch
    import paper_1709_05061_gb300 as gp
    from paper_1709_05061_gb300 import serve as S
    from paper_1709_05061_gb300 import workloads as W
    gp.build()
    torch.cuda.set_device(0)
    scale = 24
    t0 = time.perf_counter()
    st = W.rmat_stream_device(scale, 1 << 28, seed=24)
    gen_s = time.perf_counter() - t0
    reserve = 70_000_000
    window = st.numel() - reserve
    V = 1 << scale
    g = gp.Graph(V, leaf_size=LEAF)
    t0 = time.perf_counter()
    g.update(st[:window])
    g.status()
    load_s = time.perf_counter() - t0
    host_stream = st.cpu().numpy().view(np.uint64)
    del st
    torch.cuda.empty_cache()
    win = W.SlidingWindow(host_stream, window)
    # update-only sweep on the freshly loaded scale-24 array: device time per batch
    # from the library's events (the 4.3 GB array is far larger than L2), algorithmic
    # bytes from the batch's stats (both definitions), fraction of the measured peak
    peak = measured_hbm_peak()[0]
    sweep = []
    clk = ClockSampler(torch.cuda.current_device()).__enter__()
    for B in (100_000, 1_000_000):
        ts, ab, at = [], [], []
        for k in range(SWEEP_WARM + SWEEP_TIMED):
            ins, dels = win.slide(B // 2)
            di = torch.from_numpy(np.ascontiguousarray(ins).view(np.int64)).cuda()
            dd = torch.from_numpy(np.ascontiguousarray(dels).view(np.int64)).cuda()
            c_old = g.capacity
            hold_gpu()
            gp.gpma_profile_enable(g.h, True)
            st = g.update(di, dd, stats=True)
            p = gp.gpma_profile_read(g.h, reset=True)
            gp.gpma_profile_enable(g.h, False)
            if k >= SWEEP_WARM:
                ts.append(p["update"]["ms"])
                ab.append(st["alg_bytes"])
                at.append(alg_bytes_table(st, B, c_old, g.capacity))
        sweep.append(sweep_entry(B, ts, ab, at, peak))
    clk.__exit__(None, None, None)
    budget = 2 << 30  # device memory for staging and results, split by Server.with_budget
    srv = S.Server.with_budget(g, budget, max_inflight=2, keep_results=False)
    n = a.serve_requests
    # warm-up (graph capture for every batch size bucket, first analytics calls)
    srv.run(S.make_requests(60, V, win, rate=1.0, seed=100), realtime=False)
    out = {"workload": f"R-MAT scale 24 (.57/.19/.19/.05, 2^28 samples, seed 24, device-generated), "
                       f"{window} edges resident, capacity {g.capacity} slots; requests: Poisson, updates "
                       f"log-uniform 1e2..1e5 (50/50) : queries (BFS / CC / PageRank-10) = 4 : 1",
           "generate_s": gen_s, "bulk_load_s": load_s, "requests_per_run": n, "hbm_budget_bytes": budget,
           "max_batch_keys": srv.max_batch_keys, "result_slots": len(srv.d_res)}
    out["update_sweep_scale24"] = sweep
    out["update_sweep_clocks"] = clk.summary()
    clk = ClockSampler(torch.cuda.current_device()).__enter__()
    cap = srv.run(S.make_requests(n, V, win, rate=1.0, seed=101), realtime=False)
    out["closed_loop"] = cap
    # the plain path on the same kind of stream: one request at a time, nothing
    # coalesced or overlapped
    plain = S.Server(g, max_batch_keys=1 << 20, result_slots=1, max_inflight=1, coalesce=False, keep_results=False)
    out["plain_closed_loop"] = plain.run(S.make_requests(n, V, win, rate=1.0, seed=101), realtime=False)
    out["served_vs_plain_requests_per_s"] = cap["requests_per_s"] / out["plain_closed_loop"]["requests_per_s"]
    for frac in (0.5, 0.8, 0.95):
        rate = frac * cap["requests_per_s"]
        r = srv.run(S.make_requests(n, V, win, rate=rate, seed=102 + int(frac * 100)), realtime=True)
        r["offered_rate_per_s"] = rate
        out[f"load_{int(frac * 100)}"] = r
    clk.__exit__(None, None, None)
    out["serve_clocks"] = clk.summary()
    out["check"] = g.check()
    g.close()
    return out


# ---- small runs for ncu --------------------------------------------------------------------------------
def profile_case(a):
    """Load the window (R-MAT scale --scale, --window edges: 268 MB at the defaults,
    larger than the L2, a few GB on the device in all), apply one batch of --batch
    updates (graph capture, work arrays), then run one call of the case --repeat
    times, so that ncu can capture a handful of launches with few before them."""
    import torch
    import paper_1709_05061_gb300 as gp
    from paper_1709_05061_gb300 import workloads as W
    gp.build()
    torch.cuda.set_device(0)
    half = a.batch // 2
    if a.graph == "chunglu":
        return profile_case_chunglu(a)
    if a.scale >= 22:  # large graphs: drawn on the device (2^(scale+4) samples), window = all but the slides
        st = W.rmat_stream_device(a.scale, 1 << (a.scale + 4), seed=a.seed)
        stream = st.cpu().numpy().view(np.uint64)
        del st
        win = W.SlidingWindow(stream, stream.size - half * (a.repeat + 1))
    else:
        stream = W.rmat_stream(a.scale, a.window + half * (a.repeat + 1), seed=a.seed, samples=(1 << a.scale) * 16)
        win = W.SlidingWindow(stream, a.window)

    def dev(x):
        return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda()
    g = gp.Graph(1 << a.scale, leaf_size=LEAF, push_pagerank=a.push_pagerank, plain_search=a.plain_search)
    g.update(dev(win.initial), None)
    ins, dels = win.slide(half)
    g.update(dev(ins), dev(dels))
    g.status()
    torch.cuda.synchronize()
    for _ in range(a.repeat):
        if a.profile_case == "pr":
            g.pagerank(PR_ITERS, DAMPING)
        elif a.profile_case == "update":
            ins, dels = win.slide(half)
            g.update(dev(ins), dev(dels))
        elif a.profile_case == "bfs":
            g.bfs(bfs_source(stream))
        else:
            g.cc()
    g.status()
    torch.cuda.synchronize()
    out = {"profile_case": a.profile_case, "capacity": g.capacity, "check": g.check()}
    g.close()
    return out


def profile_case_chunglu(a):
    """The learned-search study's graph and batches, for ncu: load, one warm-up
    batch, then --repeat batches."""
    import torch
    import paper_1709_05061_gb300 as gp
    from paper_1709_05061_gb300 import workloads as W
    gp.build()
    torch.cuda.set_device(0)
    V, E0 = 1_600_000, 30_000_000
    n_ins = int(a.batch * 0.7)
    n_del = a.batch - n_ins
    stream = W.chung_lu_stream(V, E0 + (a.repeat + 1) * n_ins, gamma=2.1, seed=7)
    rng = np.random.default_rng(7)

    def dev(x):
        return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda()
    g = gp.Graph(V, leaf_size=LEAF, plain_search=a.plain_search)
    g.update(dev(stream[:E0]), None)
    for i in range(a.repeat + 1):
        ins = stream[E0 + i * n_ins: E0 + (i + 1) * n_ins]
        dels = stream[rng.choice(E0, n_del, replace=False)]  # live: the first E0 edges are never deleted twice here
        g.update(dev(ins), dev(dels))
    g.status()
    torch.cuda.synchronize()
    out = {"profile_case": "update", "graph": "chunglu", "capacity": g.capacity, "check": g.check()}
    g.close()
    return out


# ---- the oracle (CPU) --------------------------------------------------------------------------------
def run_oracle(a, stream, steps, max_seconds=None, skip=0):
    import oracle
    from paper_1709_05061_gb300 import workloads as W
    win = W.SlidingWindow(stream, a.window)
    o = oracle.OraclePMA(1 << a.scale, L=LEAF)
    o.update(win.initial)
    src = bfs_source(stream)
    half = a.batch // 2
    for _ in range(skip):  # untimed warm-up steps
        ins, dels = win.slide(half)
        o.update(ins, dels)
        o.pagerank(PR_ITERS, DAMPING)
        o.bfs(src)
        o.cc()
    done, t_total = 0, 0.0
    for i in range(steps):
        ins, dels = win.slide(half)
        t0 = time.perf_counter()
        o.update(ins, dels)
        o.pagerank(PR_ITERS, DAMPING)
        o.bfs(src)
        o.cc()
        t_total += time.perf_counter() - t0
        done += 1
        if max_seconds is not None and t_total >= max_seconds:
            break
    return {"value": a.batch * done / t_total, "unit": "edge updates/s", "cores": 1, "kind": "oracle",
            "sample": f"{done} full steps (update of {a.batch} + PageRank-{PR_ITERS} + BFS + CC) on the "
                      f"{a.window}-edge window, single-threaded C oracle", "seconds": t_total, "steps_done": done}


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cfg = workload_config(a, world)

    if a.profile_case:
        print(json.dumps(profile_case(a)), flush=True)
        return 0
    if a.learned_study:
        print(json.dumps({"learned_study": learned_study(a)}), flush=True)
        return 0
    if a.many_study:
        print(json.dumps({"many_study": many_study(a)}), flush=True)
        return 0
    if a.serve_study:
        print(json.dumps({"serve_study": serve_study(a)}), flush=True)
        return 0

    if a.impl == "reference":
        if rank != 0:
            return 0
        stream = make_stream(a, 0, reference=True)
        # every step is a whole oracle step (~2 s on one core); at most ~150 s of timed work
        r = run_oracle(a, stream, a.steps, skip=min(a.warmup, 3), max_seconds=150.0)
        line = {"metric": METRIC, "value": r["value"], "unit": "edge updates/s", "n_gpus": a.gpus,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * r["seconds"] / r["steps_done"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
                "data": "synthetic", "config": cfg, "impl": "reference",
                "cpu_baseline": {k: r[k] for k in ("value", "unit", "cores", "kind", "sample")},
                "e2e": {"value": r["value"], "unit": "edge updates/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0

    import torch
    dist = None
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
        dist = tdist
    else:
        torch.cuda.set_device(0)
    stream = make_stream(a, rank)
    out = run_gpu(a, stream, rank, world, dist)
    ms = out["ms_total"]
    value = job_value(world, a.batch, a.steps, ms)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "edge updates/s", "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u64", "data": "synthetic", "config": cfg,
                "gpu_launches": out["launches"], "roofline": out["roofline"], "clocks": out["clocks"],
                "phases_ms_per_step": {k: v["ms"] / PROFILED_STEPS for k, v in out["profile"].items()},
                "profiled_ms_per_step": out["profiled_ms_per_step"],
                "capacity_slots": out["capacity"], "analytics": out["analytics"]}
        if "e2e" in out:
            line["e2e"] = out["e2e"]
        if "sweep" in out:
            line["sweep"] = out["sweep"]
        if world == 1 and not a.no_cpu_baseline:
            line["cpu_baseline"] = run_oracle(a, stream, 100, max_seconds=15.0)
        if world == 1 and not a.no_studies:
            # the other configurations on the same GPU, each against the plain path
            for key, fn in (("scale24", serve_study), ("learned", learned_study), ("many", many_study)):
                t0 = time.perf_counter()
                try:
                    line[key] = fn(a)
                except Exception as e:  # a study that fails is reported, not fatal to the line
                    line[key] = {"error": f"{type(e).__name__}: {e}"}
                line[key]["wall_s"] = time.perf_counter() - t0
                torch.cuda.empty_cache()
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
