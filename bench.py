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
sys.path.insert(0, ROOT)

SCALE, WINDOW, LEAF = 20, 16_000_000, 64
SWEEP = (100, 1000, 10_000, 100_000, 1_000_000)
SWEEP_WARM, SWEEP_TIMED = 3, 10
PR_ITERS, DAMPING = 20, 0.85
METRIC = "edge updates/sec vs batch size (+HBM GB/s frac); p50/p99 update+query latency"
L2_BYTES = 129 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpma", choices=["gpma", "reference"])
    ap.add_argument("--batch", type=int, default=1_000_000)
    ap.add_argument("--scale", type=int, default=SCALE)
    ap.add_argument("--window", type=int, default=WINDOW)
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--seed", type=int, default=1)
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
    }


def stream_needed(a, reference: bool):
    half = a.batch // 2
    n = a.window + half * (a.warmup + a.steps)
    if reference:
        return n
    if not a.no_e2e:
        n += half * (a.warmup + a.steps)
    if not a.no_sweep:
        n += sum((SWEEP_WARM + SWEEP_TIMED) * (b // 2) for b in SWEEP)
    return n


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
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.p = None
        return self

    def _read(self):
        for line in self.p.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
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


def measured_hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


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

    g = gp.Graph(V, leaf_size=LEAF)
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
            times, algb, rb_times = [], [], []
            for it in range(SWEEP_WARM + SWEEP_TIMED):
                ins, dels = win.slide(b // 2)
                di, dd = to_dev(ins), to_dev(dels)
                flush.zero_()
                gp.gpma_profile_enable(g.h, True)
                s = g.update(di, dd, stats=True)
                p = gp.gpma_profile_read(g.h, reset=True)
                gp.gpma_profile_enable(g.h, False)
                ms = p["update"]["ms"]
                # sort-and-rebuild CSR baseline on the same batch
                flush.zero_()
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
                    rb_times.append(e0.elapsed_time(e1))
            med = statistics.median(times)
            gbs = statistics.median([x / (t * 1e-3) / 1e9 for x, t in zip(algb, times)])
            sweep.append({
                "batch": b, "updates_per_s": b / (med * 1e-3),
                "p50_ms": med, "p99_ms": float(np.percentile(times, 99)),
                "alg_GBps": gbs, "hbm_frac": gbs / peak,
                "rebuild_p50_ms": statistics.median(rb_times),
                "speedup_vs_rebuild": statistics.median(rb_times) / med,
            })
        out["sweep"] = sweep
        del live
    # the sweep slid only rank 0's window; every rank now continues from its own state

    ins_all, del_all = [], []
    for _ in range(a.warmup + a.steps):
        ins, dels = win.slide(half)
        ins_all.append(to_dev(ins))
        del_all.append(to_dev(dels))
    rank_t = torch.empty(V, dtype=torch.float32, device=dev)
    depth = torch.empty(V, dtype=torch.int32, device=dev)
    label = torch.empty(V, dtype=torch.int32, device=dev)

    def step(i):
        gp.gpma_update_batch(g.h, ins_all[i], del_all[i])
        gp.gpma_pagerank(g.h, PR_ITERS, DAMPING, rank_t)
        gp.gpma_bfs(g.h, src, depth)
        gp.gpma_cc(g.h, label)

    for i in range(a.warmup):
        step(i)
    gp.gpma_status(g.h)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    gp.gpma_profile_read(g.h, reset=True)
    gp.gpma_profile_enable(g.h, True)
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
    gp.gpma_profile_enable(g.h, False)
    prof = gp.gpma_profile_read(g.h, reset=True)
    gp.gpma_status(g.h)
    ms = e0.elapsed_time(e1)
    if dist:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    out["ms_total"] = ms
    out["launches"] = launches
    out["profile"] = prof
    out["clocks"] = clk.summary()
    out["capacity"] = g.capacity
    C, Vn = g.capacity, V
    # dominant kernel by device time inside the timed region
    pr = prof["pr_scatter"]
    per_launch_ms = pr["ms"] / max(pr["count"], 1)
    alg_pr = 8 * C + 20 * Vn  # stream every slot; read contrib, read+write the FP64 sum once per vertex
    out["roofline"] = {
        "kernel": "k_pr_scatter (PageRank push pass over the gapped array)",
        "bound": "hbm", "achieved": alg_pr / (per_launch_ms * 1e-3) / 1e9, "peak": peak,
        "peak_kind": peak_kind, "unit": "GB/s",
        "frac": alg_pr / (per_launch_ms * 1e-3) / 1e9 / peak,
        "traffic": None, "alg_bytes_per_launch": alg_pr, "launch_ms": per_launch_ms,
        "share_of_step": pr["ms"] / ms if ms else None,
    }

    # -- e2e: host (pinned) inputs copied in and results copied out every step ---------------------
    if not a.no_e2e:
        h_ins, h_del = [], []
        for _ in range(a.warmup + a.steps):
            ins, dels = win.slide(half)
            h_ins.append(torch.from_numpy(np.ascontiguousarray(ins).view(np.int64)).pin_memory())
            h_del.append(torch.from_numpy(np.ascontiguousarray(dels).view(np.int64)).pin_memory())
        d_ins = torch.empty(half, dtype=torch.int64, device=dev)
        d_del = torch.empty(half, dtype=torch.int64, device=dev)
        o_rank = torch.empty(V, dtype=torch.float32).pin_memory()
        o_depth = torch.empty(V, dtype=torch.int32).pin_memory()
        o_label = torch.empty(V, dtype=torch.int32).pin_memory()

        def e2e_step(i):
            d_ins.copy_(h_ins[i], non_blocking=True)
            d_del.copy_(h_del[i], non_blocking=True)
            step_io = gp.gpma_update_batch(g.h, d_ins, d_del)
            del step_io
            gp.gpma_pagerank(g.h, PR_ITERS, DAMPING, rank_t)
            gp.gpma_bfs(g.h, src, depth)
            gp.gpma_cc(g.h, label)
            o_rank.copy_(rank_t, non_blocking=True)
            o_depth.copy_(depth, non_blocking=True)
            o_label.copy_(label, non_blocking=True)
            torch.cuda.current_stream().synchronize()

        for i in range(a.warmup):
            e2e_step(i)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record()
        for i in range(a.warmup, a.warmup + a.steps):
            e2e_step(i)
        f1.record()
        torch.cuda.synchronize()
        wall = (time.perf_counter() - t0) * 1e3
        ems = max(f0.elapsed_time(f1), wall)
        if dist:
            t = torch.tensor([ems], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ems = float(t.item())
        out["e2e"] = {"value": world * a.batch * a.steps / (ems * 1e-3), "unit": "edge updates/s",
                      "h2d_bytes_per_step": 2 * half * 8, "d2h_bytes_per_step": 3 * 4 * V,
                      "ms_per_step": ems / a.steps}
        gp.gpma_status(g.h)
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
                      f"{a.window}-edge window, single-threaded C oracle", "seconds": t_total}


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cfg = workload_config(a, world)

    if a.impl == "reference":
        if rank != 0:
            return 0
        stream = make_stream(a, 0, reference=True)
        r = run_oracle(a, stream, a.steps, skip=a.warmup)
        line = {"metric": METRIC, "value": r["value"], "unit": "edge updates/s", "n_gpus": a.gpus,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * r["seconds"] / a.steps,
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
    value = world * a.batch * a.steps / (ms * 1e-3)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "edge updates/s", "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u64", "data": "synthetic", "config": cfg,
                "gpu_launches": out["launches"], "roofline": out["roofline"], "clocks": out["clocks"],
                "phases_ms_per_step": {k: v["ms"] / a.steps for k, v in out["profile"].items()},
                "capacity_slots": out["capacity"]}
        if "e2e" in out:
            line["e2e"] = out["e2e"]
        if "sweep" in out:
            line["sweep"] = out["sweep"]
        if world == 1 and not a.no_cpu_baseline:
            line["cpu_baseline"] = run_oracle(a, stream, 100, max_seconds=15.0)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
