"""Small, self-contained runs of one hot kernel family for profilers.

    python -m paper_1709_05061_gb300.profile_case --case pr      # PageRank: bucketing + 20 sum passes
    python -m paper_1709_05061_gb300.profile_case --case pr --push  # PageRank by the push pass
    python -m paper_1709_05061_gb300.profile_case --case update  # one batch of --batch updates
    python -m paper_1709_05061_gb300.profile_case --case bfs
    python -m paper_1709_05061_gb300.profile_case --case cc

Each loads an R-MAT window (default scale 20, 16,000,000 edges: a 268 MB array, larger
than the 129 MB L2, a few GB on the device in all), then runs the case once, so a
profiler can capture a handful of launches with few launches before them.  Set
GPMA_NO_GRAPHS=1 to launch every kernel of an update directly (profilers then list
each launch; the results are the same)."""
from __future__ import annotations

import argparse

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", choices=["pr", "update", "bfs", "cc"], default="pr")
    ap.add_argument("--scale", type=int, default=20)
    ap.add_argument("--window", type=int, default=16_000_000)
    ap.add_argument("--batch", type=int, default=1_000_000)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--push", action="store_true", help="PageRank by the push pass over the slots")
    a = ap.parse_args()
    import torch

    import paper_1709_05061_gb300 as gp
    from paper_1709_05061_gb300 import workloads as W
    gp.build()
    torch.cuda.set_device(0)
    half = a.batch // 2
    stream = W.rmat_stream(a.scale, a.window + half * (a.repeat + 1), seed=1, samples=(1 << a.scale) * 16)
    win = W.SlidingWindow(stream, a.window)

    def dev(x):
        return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda()
    g = gp.Graph(1 << a.scale, leaf_size=64, push_pagerank=a.push)
    g.update(dev(win.initial), None)
    ins, dels = win.slide(half)
    g.update(dev(ins), dev(dels))  # first batch of this size: graph capture, work arrays
    g.status()
    torch.cuda.synchronize()
    for _ in range(a.repeat):
        if a.case == "pr":
            g.pagerank(20, 0.85)
        elif a.case == "update":
            ins, dels = win.slide(half)
            g.update(dev(ins), dev(dels))
        elif a.case == "bfs":
            g.bfs(int(stream[0] >> np.uint64(32)))
        else:
            g.cc()
    g.status()
    torch.cuda.synchronize()
    print("ok", a.case, g.capacity)


if __name__ == "__main__":
    main()
