"""GPU parity of the sharded census: for every shard count, the accumulators
of tc_census_shard summed over the shards (int64 sums, wrapping like the
library's uint64 words) and folded by tc_census_fold equal the oracle's
census, on both triangle paths, under exact-cost binning, with per-row task
terms, and for a mixed batch routed per graph.  One GPU runs all shards one
after the other: each shard is a whole census pipeline with a share of the
work, so this is the computation each process of a sharded run makes."""
import numpy as np
import pytest

import oracle
import synth
import paper_1603_02655_b300 as tc
from paper_1603_02655_b300 import build as tcbuild

pytestmark = pytest.mark.gpu

MERGE, FWD, AUTO = tc.TC_TRI_MERGE, tc.TC_TRI_FORWARD, tc.TC_TRI_AUTO
CONFIGS = {
    "auto": dict(),
    "fwd": dict(tri_path=FWD),
    "fwd_map_all": dict(tri_path=FWD, fwd_big=1),
    "fwd_rows": dict(tri_path=FWD, row_tasks=1),
    "merge": dict(tri_path=MERGE),
    "merge_no_owner": dict(tri_path=MERGE, own_min=0, thr_thread=16, thr_warp=96),
    "merge_rows": dict(tri_path=MERGE, row_tasks=1),
    "exact": dict(tri_path=MERGE, bin_mode=tc.TC_BIN_EXACT, own_min=0),
}


@pytest.fixture(scope="module", autouse=True)
def lib(cuda_ok):
    tcbuild.build()
    return tc.load()


def sharded(gs, nshards, opts):
    import torch
    total = torch.zeros(tc.TC_ACC_WORDS * len(gs), dtype=torch.int64, device="cuda")
    acc = torch.empty_like(total)
    for k in range(nshards):
        acc.fill_(-1)  # every word is overwritten
        tc.tc_census_shard(gs, k, nshards, acc, opts)
        total += acc
    return tc.tc_census_fold(gs, total)


def hub_graph(rng, n, hubs, hub_deg, extra, recip):
    src, dst = [], []
    for h in range(hubs):
        nb = rng.choice(n, size=hub_deg, replace=False)
        out = rng.random(hub_deg) < 0.5
        src.append(np.where(out, h, nb))
        dst.append(np.where(out, nb, h))
    src.append(rng.integers(0, n, extra))
    dst.append(rng.integers(0, n, extra))
    s = np.concatenate(src).astype(np.int32)
    d = np.concatenate(dst).astype(np.int32)
    rec = rng.random(s.size) < recip
    return np.concatenate([s, d[rec]]), np.concatenate([d, s[rec]])


@pytest.mark.parametrize("seed", range(2))
def test_shards_of_one_graph_sum_to_the_census(seed):
    rng = np.random.default_rng(1200 + seed)
    n = 12_000
    src, dst = hub_graph(rng, n, 3, int(rng.integers(1500, 4000)), 60_000, 0.25)
    want = oracle.census(n, src, dst, threads=8)
    g = tc.tc_graph_build(n, src, dst)
    try:
        for name, kw in CONFIGS.items():
            o = tc.tc_opts_default(**kw)
            for nshards in (1, 2, 3, 7):
                assert sharded([g], nshards, o) == [want], (name, nshards)
    finally:
        tc.tc_graph_free(g)


def test_shards_of_a_mixed_batch_sum_to_each_census():
    """Graphs of both paths in one call (per-graph routing), more shards than
    some graphs have rows, and a graph whose 003 count needs 128 bits."""
    rng = np.random.default_rng(77)
    arcs, ns = [], []
    for i in range(9):
        if i % 2:
            n = int(rng.integers(2000, 5000))
            s_, d_ = hub_graph(rng, n, 2, int(rng.integers(400, 1200)), 4 * n, 0.2)
        else:
            n = int(rng.integers(5, 300))
            a = synth.gnp(n, 0.05, recip=0.3, seed=int(rng.integers(1 << 30)))
            s_, d_ = a.src, a.dst
        arcs.append((s_, d_))
        ns.append(n)
    n_big = 5_000_000
    arcs.append((np.array([0, 1, 2], np.int32), np.array([1, 2, 0], np.int32)))
    ns.append(n_big)
    want = [oracle.census(n, a[0], a[1]) for n, a in zip(ns, arcs)]
    assert want[-1][0] >= 1 << 64
    off = np.cumsum([0] + [a[0].size for a in arcs])
    gs = tc.tc_graph_build_batched(ns, off, np.concatenate([a[0] for a in arcs]).astype(np.int32),
                                   np.concatenate([a[1] for a in arcs]).astype(np.int32))
    try:
        assert set(tc.tc_path_route(gs[:-1])) == {FWD, MERGE}
        for name in ("auto", "fwd", "merge", "exact"):
            o = tc.tc_opts_default(**CONFIGS[name])
            for nshards in (1, 2, 5, 16):
                assert sharded(gs, nshards, o) == want, (name, nshards)
            # a shuffled subset keeps each result with its own graph
            order = [7, 2, 9, 0]
            assert sharded([gs[i] for i in order], 3, o) == [want[i] for i in order], name
    finally:
        for g in gs:
            tc.tc_graph_free(g)


def test_sharded_helpers_on_a_one_process_group(tmp_path):
    """census_sharded (shard + all-reduce + fold) and census_graph_shards
    (whole graphs + gather) through a gloo group of one process: the CUDA
    accumulators go through a host copy for the gloo sum."""
    import torch.distributed as dist
    from paper_1603_02655_b300 import shard
    arcs = [synth.gnp(200 + 50 * k, 0.03, recip=0.2, seed=40 + k) for k in range(4)]
    want = [oracle.census(a.n, a.src, a.dst) for a in arcs]
    off = np.cumsum([0] + [a.src.size for a in arcs])
    gs = tc.tc_graph_build_batched([a.n for a in arcs], off, np.concatenate([a.src for a in arcs]),
                                   np.concatenate([a.dst for a in arcs]))
    dist.init_process_group("gloo", init_method=f"file://{tmp_path}/pg", rank=0, world_size=1)
    try:
        assert shard.census_sharded(gs, 0, 1) == want
        assert shard.census_graph_shards(gs, [a.src.size for a in arcs], 0, 1) == want
    finally:
        dist.destroy_process_group()
        for g in gs:
            tc.tc_graph_free(g)


def test_shard_arguments_are_checked():
    import torch
    g = tc.tc_graph_build(4, np.array([0, 1], np.int32), np.array([1, 2], np.int32))
    try:
        acc = torch.zeros(tc.TC_ACC_WORDS, dtype=torch.int64, device="cuda")
        for k, n in ((0, 0), (2, 2), (-1, 3)):
            with pytest.raises(tc.TcError) as e:
                tc.tc_census_shard([g], k, n, acc)
            assert e.value.status == tc.TC_ERR_ARG
        with pytest.raises(tc.TcError):
            tc.tc_census_shard([g], 0, 1, acc[:10])
        with pytest.raises(tc.TcError):
            tc.tc_census_shard([g], 0, 1, acc.cpu())
    finally:
        tc.tc_graph_free(g)
