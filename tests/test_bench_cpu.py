"""bench.py's host logic on CPU: the reference arm (the CPU oracle) and the
multi-rank path under torch.distributed with the gloo backend."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def bench_unit():
    sys.path.insert(0, ROOT)
    import bench
    return bench.UNIT


def test_reference_arm_prints_one_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "c1", "--steps", "3",
                        "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == bench_unit()
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_two_ranks_gloo():
    env = dict(os.environ, MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(free_port()), "bench.py", "--impl",
                        "reference", "--workload", "c1", "--gpus", "2", "--steps", "3", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1  # rank 0 alone prints
    assert json.loads(lines[0])["n_gpus"] == 2


def _max_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    q.put((rank, bench.max_over_ranks(10.0 + rank, dist)))
    bench.barrier(dist)
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_max_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = dict(q.get() for _ in range(2))
    assert res == {0: 11.0, 1: 11.0}


def test_oracle_sample_ranges_are_sized_and_bounded():
    # the CPU-baseline sample: vertex costs = merged entries charged to each
    # lower endpoint; ranges of about the target cost, heavy ones left out,
    # and a timed sample that stays near its time budget
    import time
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    import synth
    a = synth.rmat(12, 8, recip=0.1, seed=3)
    cost = bench.vertex_costs(a)
    s, d = a.src.astype(np.int64), a.dst.astype(np.int64)
    keep = s != d
    u, v = np.minimum(s[keep], d[keep]), np.maximum(s[keep], d[keep])
    pairs = np.unique(u * a.n + v)
    deg = np.bincount(pairs // a.n, minlength=a.n) + np.bincount(pairs % a.n, minlength=a.n)
    assert cost.sum() == float((deg.astype(np.int64) ** 2).sum())  # sum over dyads of d_u + d_v
    rng = np.random.default_rng(0)
    target, cap = cost.sum() / 50, cost.sum() / 10
    ranges, skipped = bench.cost_ranges(cost, target, cap, rng)
    covered = np.zeros(a.n, bool)
    for lo, hi, c in ranges:
        assert 0 <= lo < hi <= a.n and 0 < c <= cap
        assert abs(c - cost[lo:hi].sum()) < 1e-6 * max(1.0, c)
        assert not covered[lo:hi].any()
        covered[lo:hi] = True
    every, none = bench.cost_ranges(cost, target, float("inf"), np.random.default_rng(0))
    assert none == 0 and skipped == sum(1 for r in every if r[2] > cap)
    assert len(ranges) + skipped == len(every)
    t = time.perf_counter()
    rate, threads, verts, ents, wall, _ = bench.oracle_sample_rate(a, 1.0, threads=2, cost=cost)
    assert rate > 0 and ents > 0 and verts > 0 and threads == 2
    assert time.perf_counter() - t < 60
