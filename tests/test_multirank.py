"""The multi-rank logic of bench.py on CPU with two gloo ranks: each rank gets
its own replica stream (replicas only, weak scaling), the job time is the
maximum over ranks, the job value counts every rank's updates, and under
--impl reference only rank 0 prints."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        _body(rank, world, dist, q, bench)
    except Exception as e:  # report instead of leaving the parent waiting
        q.put((rank, repr(e), None, None))
    finally:
        dist.destroy_process_group()


def _body(rank, world, dist, q, bench):
    ms = 10.0 + 5.0 * rank                     # rank 1 is the slower one
    job_ms = bench.max_over_ranks(ms, dist, "cpu")

    class A:
        scale, window, batch, steps, warmup, seed = 8, 2000, 100, 3, 3, 1
    st = bench.make_stream(A, rank, reference=True)
    q.put((rank, job_ms, bench.job_value(world, A.batch, A.steps, job_ms), st[:50].tolist()))


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, v0, s0), (r1, ms1, v1, s1) = out
    assert ms0 == ms1 == 15.0                      # the max over ranks, on every rank
    assert v0 == v1 == pytest.approx(2 * 100 * 3 / 15e-3)
    assert s0 != s1                                # differently seeded replicas
    assert len(set(s0)) == len(s0)


def test_reference_arm_prints_on_rank0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--scale", "8", "--window", "2000", "--batch", "100", "--steps", "3"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--scale", "8", "--window", "2000", "--batch", "100", "--steps", "3"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert np.isfinite(line["e2e"]["value"])
