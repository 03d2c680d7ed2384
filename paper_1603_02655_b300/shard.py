"""Spreading a census over several processes (one GPU each).

The thesis names a multi-GPU system as future work (Ch. 6, "Future work").
The census shards without any exchange on the data path: every canonical
dyad's contributions are independent (Sec. 2.2), so the only communication
is a sum of the per-graph accumulators (or, for whole graphs per process,
a gather of the 17-word results).  Two ways:

* one graph (or one batch) cut into shards: every process builds its own
  replica of the graph from the arc list, runs `tc_census_shard` for its
  shard, the raw accumulators (TC_ACC_WORDS words per graph) are summed over
  the processes (`allreduce_words`), and `tc_census_fold` closes the census;
* whole graphs per process (many independent graphs, as in a batch):
  `graph_shares` deals the graphs out by cost, each process censuses its
  share, and `gather_results` sums the zero-padded result tables.

The sums are word-wise modulo 2^64 (int64 tensors wrap like the library's
uint64 words); collectives run on a torch.distributed process group (NCCL on
CUDA tensors, or gloo through host memory).
"""
from __future__ import annotations

import heapq

import numpy as np

from . import TC_ACC_WORDS, tc_census_batched, tc_census_fold, tc_census_shard


def graph_shares(costs, world: int) -> list[list[int]]:
    """Whole graphs per process: indices of the graphs each of `world`
    processes takes, dealt largest cost first to the least loaded process
    (longest-processing-time rule; ties by process index).  Every graph goes
    to exactly one process; each list is in increasing index order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = np.asarray(costs, dtype=np.float64)
    order = sorted(range(costs.size), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    shares: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shares[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(s) for s in shares]


def allreduce_words(t, group=None):
    """Sum an int64 tensor over the processes of `group` in place (wrapping).
    CUDA tensors go through the group's backend when it is NCCL; otherwise
    through a host copy (gloo)."""
    import torch.distributed as dist
    if t.is_cuda and dist.get_backend(group) != "nccl":
        h = t.cpu()
        dist.all_reduce(h, op=dist.ReduceOp.SUM, group=group)
        t.copy_(h)
    else:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def census_sharded(gs, rank: int, world: int, group=None, opts=None, stream=None):
    """The census of graphs `gs` (handles of one build, the same graphs in
    every process) computed as shard `rank` of `world` here and summed over
    the group: returns the per-graph censuses (host lists) in every process."""
    import torch
    acc = torch.zeros(TC_ACC_WORDS * max(len(gs), 1), dtype=torch.int64, device="cuda")
    tc_census_shard(gs, rank, world, acc, opts=opts, stream=stream)
    torch.cuda.synchronize()
    allreduce_words(acc, group)
    return tc_census_fold(gs, acc, stream=stream)


def gather_results(rows: dict[int, list[int]], G: int, group=None) -> list[list[int]]:
    """Every process's census rows ({graph index: 16 counts}) merged into the
    full table of G graphs in every process: a zero-padded [G][17] int64
    table (16 counts as 64-bit words, then the high word of 003) summed over
    the group.  A graph must be censused by exactly one process."""
    import torch
    t = torch.zeros((max(G, 1), 17), dtype=torch.int64)
    for i, c in rows.items():
        w = [int(x) for x in c]
        words = [x & ((1 << 64) - 1) for x in w] + [w[0] >> 64]
        t[i] = torch.tensor([x - (1 << 64) if x >= 1 << 63 else x for x in words], dtype=torch.int64)
    allreduce_words(t, group)
    out = []
    for i in range(G):
        words = [int(x) & ((1 << 64) - 1) for x in t[i].tolist()]
        out.append([words[0] | (words[16] << 64)] + words[1:16])
    return out


def census_graph_shards(gs, costs, rank: int, world: int, group=None, opts=None, stream=None):
    """Whole graphs per process: this process censuses its share of `gs`
    (graph_shares by `costs`) in one batched call; the results of all
    processes are gathered.  Returns every graph's census in every process."""
    mine = graph_shares(costs, world)[rank]
    res = tc_census_batched([gs[i] for i in mine], opts, stream=stream) if mine else []
    return gather_results(dict(zip(mine, res)), len(gs), group)
