"""Host logic of the sharded census, on CPU: the whole-graph partition, and
the sums over processes (two gloo ranks) of shard results, with the oracle
standing in for each process's GPU census.

* One graph cut into shards: each rank takes the canonical dyads whose lower
  endpoint lies in its half of the vertex range (the oracle's range census,
  types 1..15 without the 003 closure), the shares are summed with
  `allreduce_words` (int64 words, wrapping), and 003 = C(n,3) minus the rest
  closes the census: it must equal the oracle's full census (Sec. 2.2: the
  dyads' contributions are independent and add up).
* Whole graphs per rank: `graph_shares` deals a batch out by cost, each rank
  censuses its share with the oracle, and `gather_results` must give every
  rank the full table.
"""
import os
import socket
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_graph_shares_deal_every_graph_once_and_balance():
    sys.path.insert(0, ROOT)
    from paper_1603_02655_b300.shard import graph_shares
    rng = np.random.default_rng(5)
    for world in (1, 2, 3, 8):
        costs = rng.pareto(1.5, 500) * 1e6
        sh = graph_shares(costs, world)
        assert len(sh) == world
        flat = sorted(i for s in sh for i in s)
        assert flat == list(range(costs.size))
        loads = [costs[s].sum() for s in sh]
        # longest-processing-time bound: no load exceeds the mean by more than the largest cost
        assert max(loads) <= costs.sum() / world + costs.max() + 1e-6
    assert graph_shares([], 4) == [[], [], [], []]
    assert graph_shares([3.0, 1.0, 2.0], 2) == [[0], [1, 2]]


def _graph():
    import synth
    return synth.rmat(11, 8, recip=0.2, seed=7)


def _split_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1603_02655_b300.shard import allreduce_words
    a = _graph()
    g = oracle.Graph(a.n, a.src, a.dst)
    lo, hi = rank * a.n // world, (rank + 1) * a.n // world
    part, _ = g.census_range(lo, hi)
    g.close()
    words = torch.tensor([(int(x) + (1 << 63)) % (1 << 64) - (1 << 63) for x in part], dtype=torch.int64)
    allreduce_words(words)
    total = [int(x) & ((1 << 64) - 1) for x in words.tolist()]
    total[0] = oracle.choose3(a.n) - sum(total[1:])
    q.put((rank, total))
    dist.destroy_process_group()


def _gather_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1603_02655_b300.shard import gather_results, graph_shares
    batch = _batch()
    costs = [a.src.size for _, a in batch]
    mine = graph_shares(costs, world)[rank]
    rows = {i: oracle.census(batch[i][0], batch[i][1].src, batch[i][1].dst) for i in mine}
    q.put((rank, gather_results(rows, len(batch))))
    dist.destroy_process_group()


def _batch():
    import synth
    out = []
    for k in range(7):
        a = synth.gnp(int(40 + 37 * k), 4.0 / (40 + 37 * k), recip=0.3, seed=100 + k)
        out.append((a.n, a))
    # a graph whose 003 count needs more than 64 bits
    n = 5_000_000
    out.append((n, synth.Arcs(n, np.array([0, 1], np.int32), np.array([1, 2], np.int32))))
    return out


def _run(target):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=target, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    return res


def test_two_gloo_ranks_sum_dyad_shards_to_the_census():
    sys.path.insert(0, ROOT)
    import oracle
    a = _graph()
    want = oracle.census(a.n, a.src, a.dst)
    res = _run(_split_worker)
    assert res[0] == want and res[1] == want


def test_two_gloo_ranks_gather_whole_graph_shares():
    sys.path.insert(0, ROOT)
    import oracle
    want = [oracle.census(n, a.src, a.dst) for n, a in _batch()]
    assert want[-1][0] >= 1 << 64
    res = _run(_gather_worker)
    assert res[0] == want and res[1] == want
