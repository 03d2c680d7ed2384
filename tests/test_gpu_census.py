"""GPU parity: the CUDA census against the CPU oracle, element by element
(all 16 counts, exact integers), through the C-ABI."""
import json
import os

import numpy as np
import pytest

import oracle
import synth
import paper_1603_02655_b300 as tc
from paper_1603_02655_b300 import build as tcbuild

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
THREADS = min(os.cpu_count() or 1, 32)
BIG = 1 << 30

# binning configurations: default, everything per thread, per warp, per CTA
# chunk (tiny chunks: every task split), and small mixed thresholds
MERGE, FWD = tc.TC_TRI_MERGE, tc.TC_TRI_FORWARD
BINS = {
    # the default: each graph on the path its router picks (degree-skew rule)
    "default": {},
    # forward path: owners by tag map and by binary search
    "fwd": dict(tri_path=FWD),
    "fwd_map_all": dict(tri_path=FWD, fwd_big=1),
    "fwd_search_all": dict(tri_path=FWD, fwd_big=BIG),
    "fwd_map_mid": dict(tri_path=FWD, fwd_big=4),
    "fwd_row_tasks": dict(tri_path=FWD, row_tasks=1),
    # merge path: owner lookups and merge bins
    "merge_default": dict(tri_path=MERGE),
    "no_owner": dict(tri_path=MERGE, own_min=0),
    "nostream": dict(tri_path=MERGE, stream_max=0, own_min=0),
    "stream_all": dict(tri_path=MERGE, thr_thread=0, thr_warp=0, stream_max=1024, own_min=0),
    "stream_chunks": dict(tri_path=MERGE, thr_thread=0, thr_warp=0, stream_max=1 << 30, own_min=0),
    "hub_separate": dict(tri_path=MERGE, thr_thread=0, thr_warp=0, stream_max=1 << 30, persistent=0, own_min=0),
    "thread": dict(tri_path=MERGE, thr_thread=BIG, thr_warp=BIG, own_min=0),
    "warp": dict(tri_path=MERGE, thr_thread=0, thr_warp=BIG, stream_max=0, own_min=0),
    "separate": dict(tri_path=MERGE, persistent=0, own_min=0),
    "cta": dict(tri_path=MERGE, thr_thread=0, thr_warp=0, chunk=256, split_cta=1, stream_max=0, persistent=0,
                own_min=0),
    "wtile": dict(tri_path=MERGE, thr_thread=0, thr_warp=0, chunk=256, stream_max=0, own_min=0),
    "cta_big": dict(tri_path=MERGE, thr_thread=16, thr_warp=200, chunk=3840, split_cta=1, stream_max=8,
                    persistent=0, own_min=0),
    "mixed": dict(tri_path=MERGE, thr_thread=8, thr_warp=40, chunk=512, own_min=0),
    "persistent": dict(tri_path=MERGE, persistent=1, own_min=0),
    "persistent_small": dict(tri_path=MERGE, persistent=1, thr_thread=8, thr_warp=64, chunk=256, stream_max=32,
                             own_min=0),
    "owner_all": dict(tri_path=MERGE, own_min=1),
    "owner_mid": dict(tri_path=MERGE, own_min=64, thr_thread=8, thr_warp=64),
    "owner_sep": dict(tri_path=MERGE, own_min=32, persistent=0, stream_max=0),
    "row_tasks": dict(tri_path=MERGE, row_tasks=1),
    "row_tasks_merge": dict(tri_path=MERGE, row_tasks=1, own_min=0, thr_thread=8, thr_warp=64),
    "exact": dict(tri_path=MERGE, bin_mode=tc.TC_BIN_EXACT),
    "exact_merges": dict(tri_path=MERGE, bin_mode=tc.TC_BIN_EXACT, own_min=0, thr_thread=16, thr_warp=96),
    "exact_rows": dict(tri_path=MERGE, bin_mode=tc.TC_BIN_EXACT, own_min=0, row_tasks=1, thr_thread=16,
                       thr_warp=96),
}


@pytest.fixture(scope="module", autouse=True)
def lib(cuda_ok):
    tcbuild.build()
    return tc.load()


def opts(name):
    return tc.tc_opts_default(**BINS[name])


def gpu_census(n, src, dst, o=None):
    g = tc.tc_graph_build(n, src, dst)
    try:
        return tc.tc_census(g, o)
    finally:
        tc.tc_graph_free(g)


def rand_graph(rng, n, p, r):
    s, d = np.nonzero(rng.random((n, n)) < p)
    keep = s != d
    s, d = s[keep], d[keep]
    rec = rng.random(s.size) < r
    return (np.concatenate([s, d[rec]]).astype(np.int32),
            np.concatenate([d, s[rec]]).astype(np.int32))


def hub_graph(rng, n, hubs, hub_deg, extra, recip):
    """A few hubs joined to many vertices plus random arcs: tasks of every bin."""
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


# ------------------------------------------------------------ tiny graphs

def test_all_64_triads_batched():
    T = oracle.triad_table()
    bits = {(0, 1): 1, (1, 0): 2, (0, 2): 4, (2, 0): 8, (1, 2): 16, (2, 1): 32}
    src, dst, off = [], [], [0]
    for c in range(64):
        arcs = [ab for ab, b in bits.items() if c & b]
        src += [a for a, _ in arcs]
        dst += [b for _, b in arcs]
        off.append(len(src))
    gs = tc.tc_graph_build_batched([3] * 64, off, src, dst)
    try:
        for name in BINS:
            res = tc.tc_census_batched(gs, opts(name))
            for c in range(64):
                want = [0] * 16
                want[T[c]] = 1
                assert res[c] == want, (name, c)
    finally:
        for g in gs:
            tc.tc_graph_free(g)


def test_all_4096_four_vertex_digraphs_batched():
    pairs = [(a, b) for a in range(4) for b in range(4) if a != b]
    src, dst, off, want = [], [], [0], []
    for mask in range(1 << 12):
        arcs = [pairs[k] for k in range(12) if mask >> k & 1]
        s = [a for a, _ in arcs]
        d = [b for _, b in arcs]
        src += s
        dst += d
        off.append(len(src))
        want.append(oracle.brute_census(4, s, d))
    gs = tc.tc_graph_build_batched([4] * 4096, off, src, dst)
    try:
        for name in ("default", "fwd_map_all", "fwd_search_all", "cta", "mixed"):
            assert tc.tc_census_batched(gs, opts(name)) == want, name
        # a shuffled subset keeps each result with its own graph
        rng = np.random.default_rng(3)
        pick = rng.permutation(4096)[:1000]
        sub = tc.tc_census_batched([gs[i] for i in pick])
        assert sub == [want[i] for i in pick]
    finally:
        for g in gs:
            tc.tc_graph_free(g)


def fold(codes):
    T = oracle.triad_table()
    out = [0] * 16
    for c, k in enumerate(codes):
        out[T[c]] += k
    return out


def test_codes_match_oracle():
    rng = np.random.default_rng(21)
    graphs = [(40, *rand_graph(rng, 40, 0.15, 0.3)), (300, *rand_graph(rng, 300, 0.03, 0.5)),
              (3000, *hub_graph(rng, 3000, 3, 900, 20000, 0.2))]
    for n, src, dst in graphs:
        want = oracle.census_codes(n, src, dst)
        g = tc.tc_graph_build(n, src, dst)
        try:
            for name in ("default", "fwd_map_all", "fwd_search_all", "merge_default", "owner_all", "no_owner",
                         "row_tasks", "cta", "stream_all"):
                got = tc.tc_census_codes(g, opts(name))
                assert got == want, (n, name)
                assert fold(got) == tc.tc_census(g, opts(name)), (n, name)
        finally:
            tc.tc_graph_free(g)


def test_codes_batched_all_64_triads():
    bits = {(0, 1): 1, (1, 0): 2, (0, 2): 4, (2, 0): 8, (1, 2): 16, (2, 1): 32}
    src, dst, off, want = [], [], [0], []
    for c in range(64):
        arcs = [ab for ab, b in bits.items() if c & b]
        s = [a for a, _ in arcs]
        d = [b for _, b in arcs]
        src += s
        dst += d
        off.append(len(src))
        want.append(oracle.brute_census_codes(3, s, d))
    gs = tc.tc_graph_build_batched([3] * 64, off, src, dst)
    try:
        for name in ("default", "fwd_map_all", "owner_all", "thread"):
            assert tc.tc_census_codes_batched(gs, opts(name)) == want, name
    finally:
        for g in gs:
            tc.tc_graph_free(g)


# ------------------------------------------------------------ random graphs

@pytest.mark.parametrize("seed", range(6))
def test_random_graphs_all_bins(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 400))
    p = float(rng.choice([0.005, 0.03, 0.1, 0.4]))
    r = float(rng.choice([0.0, 0.3, 1.0]))
    src, dst = rand_graph(rng, n, p, r)
    want = oracle.census(n, src, dst, threads=THREADS)
    for name in BINS:
        assert gpu_census(n, src, dst, opts(name)) == want, name


@pytest.mark.parametrize("seed", range(3))
def test_hub_graphs_span_tiles_and_chunks(seed):
    # hub tasks of |N(u)|+|N(v)| ~ 4000-9000: several 3840-entry CTA tiles,
    # split into chunks, with ragged tails
    rng = np.random.default_rng(50 + seed)
    n = 9000
    src, dst = hub_graph(rng, n, hubs=3, hub_deg=int(rng.integers(2500, 4500)), extra=30000,
                         recip=0.2)
    want = oracle.census(n, src, dst, threads=THREADS)
    for name in BINS:
        assert gpu_census(n, src, dst, opts(name)) == want, name


def test_hub_tasks_stage_short_list_in_pieces():
    # hubs of exact degrees around the 1024-entry staging limit, all joined to
    # one another: hub-hub dyads whose shorter list has 1024 entries run in the
    # stream bin, longer ones (1025, 2048, 2049, 3500) in the hub launch, which
    # stages the shorter list in 1024-entry pieces (the last one ragged)
    rng = np.random.default_rng(7)
    n = 6000
    degs = [1023, 1024, 1025, 2048, 2049, 3500]
    H = len(degs)
    src, dst = [], []
    for h, D in enumerate(degs):
        nb = np.concatenate([np.delete(np.arange(H), h),
                             rng.choice(np.arange(H, n), size=D - (H - 1), replace=False)])
        out = rng.random(nb.size) < 0.5
        src.append(np.where(out, h, nb))
        dst.append(np.where(out, nb, h))
    s = rng.integers(H, n, 20000)
    d = rng.integers(H, n, 20000)
    src.append(s)
    dst.append(d)
    src = np.concatenate(src).astype(np.int32)
    dst = np.concatenate(dst).astype(np.int32)
    want = oracle.census(n, src, dst, threads=THREADS)
    for h, D in enumerate(degs):  # |N(h)|: distinct neighbours either way
        assert np.unique(np.concatenate([dst[src == h], src[dst == h]])).size == D
    hubs = sum(1 for i in range(H) for j in range(i + 1, H) if min(degs[i], degs[j]) > 1024)
    for name in ("default", "merge_default", "no_owner", "separate", "stream_chunks", "hub_separate", "nostream"):
        o = tc.tc_opts_default(profile=1, **BINS[name])
        assert gpu_census(n, src, dst, o) == want, name
        p = tc.tc_census_profile()
        path = o.tri_path if o.tri_path != tc.TC_TRI_AUTO else route_of(n, src, dst)
        if path == tc.TC_TRI_FORWARD:  # no merge bins: every triangle from the forward lists
            assert sum(p["bin_tasks"]) == 0 and p["owner_tasks"] == 0, name
            assert p["map_triangles"] + p["search_triangles"] == triangles(want), name
        elif o.own_min > 0:  # the hubs own their dyads: looked up, not streamed
            assert p["hub_tasks"] == 0 and p["owner_tasks"] > 0, name
        elif o.stream_max > 1024:
            assert p["hub_tasks"] == hubs, name
            assert p["hub_entries"] > 0
        else:
            assert p["hub_tasks"] == 0, name


def route_of(n, src, dst):
    g = tc.tc_graph_build(n, src, dst)
    try:
        return tc.tc_path_route([g])[0]
    finally:
        tc.tc_graph_free(g)


def triangles(census):
    """Triads whose three pairs are all adjacent."""
    return sum(census[idx(t)] for t in ("030T", "030C", "120D", "120U", "120C", "210", "300"))


def forward_profile(n, src, dst, name):
    o = tc.tc_opts_default(profile=1, **BINS[name])
    c = gpu_census(n, src, dst, o)
    return c, tc.tc_census_profile()


def star_plus(rng, n, hub, leaves, extra):
    """A hub joined to `leaves` (random directions, some mutual) plus random
    arcs among the leaves."""
    out = rng.random(leaves.size) < 0.5
    mut = rng.random(leaves.size) < 0.2
    src = [np.where(out, hub, leaves), leaves[mut]]
    dst = [np.where(out, leaves, hub), np.full(mut.sum(), hub)]
    src.append(rng.choice(leaves, extra))
    dst.append(rng.choice(leaves, extra))
    return np.concatenate(src).astype(np.int32), np.concatenate(dst).astype(np.int32)


def owner_profile(n, src, dst, **over):
    o = tc.tc_opts_default(profile=1, **{"tri_path": MERGE, **over})
    c = gpu_census(n, src, dst, o)
    return c, tc.tc_census_profile()


def test_owner_staging_boundary():
    # owners of up to 512 entries are copied to shared memory, larger ones
    # are looked up in global memory: hubs of 511, 512 and 513 entries
    # over the same neighbourhood, joined to one another
    rng = np.random.default_rng(5)
    n = 20_000
    pool = np.arange(3, n)
    src, dst = [], []
    for h, D in enumerate((511, 512, 513)):
        nb = np.concatenate([np.delete(np.arange(3), h), rng.choice(pool[:12_000], D - 2, replace=False)])
        out = rng.random(nb.size) < 0.5
        src.append(np.where(out, h, nb))
        dst.append(np.where(out, nb, h))
    src.append(rng.integers(3, n, 40_000))
    dst.append(rng.integers(3, n, 40_000))
    src, dst = np.concatenate(src).astype(np.int32), np.concatenate(dst).astype(np.int32)
    want = oracle.census(n, src, dst, threads=THREADS)
    for own_min in (1, 128, 513):
        c, p = owner_profile(n, src, dst, own_min=own_min)
        assert c == want, own_min
        assert p["owner_tasks"] > 0


def test_owner_structured_ids():
    # owners whose neighbour ids share their low bits (stride 64: every key in
    # few id buckets) or are consecutive, joined to one another, plus owners
    # of 1 to 4 entries
    rng = np.random.default_rng(17)
    n = 70_000
    strided = np.arange(64, 64 * 1000, 64)
    run = np.arange(60_000, 63_000)
    src = [np.zeros(strided.size, np.int64), np.full(run.size, 1)]
    dst = [strided, run]
    for hub, nb in ((0, run[::3]), (1, strided[::2])):  # shared neighbours
        src.append(np.full(nb.size, hub))
        dst.append(nb)
    src.append([0, 5, 6, 7, 7, 9, 9, 9])
    dst.append([1, 6, 7, 5, 8, 10, 11, 12])
    src.append(rng.integers(2, n, 30_000))
    dst.append(rng.integers(2, n, 30_000))
    src, dst = np.concatenate(src).astype(np.int32), np.concatenate(dst).astype(np.int32)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    flip = rng.random(src.size) < 0.3
    src, dst = np.where(flip, dst, src), np.where(flip, src, dst)
    want = oracle.census(n, src, dst, threads=THREADS)
    for own_min in (1, 128):
        c, p = owner_profile(n, src, dst, own_min=own_min)
        assert c == want, own_min
        assert p["owner_tasks"] > 0


def test_owner_large_and_skewed():
    # owners above 512 entries keep only 32-bit bucket starts in shared
    # memory and read their list from global memory; two such hubs share
    # neighbours (their dyad has both lists large)
    rng = np.random.default_rng(11)
    n = 200_000
    leaves = rng.choice(n - 1, 40_000, replace=False)
    s1, d1 = star_plus(rng, n, n - 1, leaves, 60_000)
    leaves2 = np.concatenate([rng.choice(leaves, 10_000, replace=False),
                              rng.choice(n - 1, 10_000, replace=False)])
    leaves2 = np.unique(leaves2[leaves2 != 7])
    s2, d2 = star_plus(rng, n, 7, leaves2, 0)
    src, dst = np.concatenate([s1, s2, [7]]), np.concatenate([d1, d2, [n - 1]])
    want = oracle.census(n, src, dst, threads=THREADS)
    for own_min in (1, 1000, 20000):
        c, p = owner_profile(n, src, dst, own_min=own_min)
        assert c == want, own_min
        assert p["owner_items"] >= 1 and p["owner_tasks"] > 0
    for name in ("fwd", "fwd_map_all", "fwd_search_all"):  # both lookup forms in one graph
        c, p = forward_profile(n, src, dst, name)
        assert c == want, name
        assert p["map_triangles"] + p["search_triangles"] == triangles(want), name
    # an owner whose neighbours all have small ids: they crowd into a few id
    # buckets (long scans), which must stay exact
    n = 1_000_000
    s3, d3 = star_plus(rng, n, n - 1, np.arange(20_000), 50_000)
    want = oracle.census(n, s3, d3, threads=THREADS)
    c, p = owner_profile(n, s3, d3, own_min=1)
    assert c == want
    # with own_min = 1 every dyad is an owner task
    assert p["owner_tasks"] == oracle.Graph(n, s3, d3).stats()["dyads"]
    assert sum(p["bin_tasks"]) == 0


def test_c1_matches_golden_and_brute():
    a = synth.c1()
    gold = json.load(open(os.path.join(GOLDEN, "census_c1.json")))["census"]
    assert oracle.brute_census(a.n, a.src, a.dst) == gold
    for name in BINS:
        assert gpu_census(a.n, a.src, a.dst, opts(name)) == gold, name


# ------------------------------------------------------------ closed forms

def C3(n):
    return n * (n - 1) * (n - 2) // 6


def idx(name):
    return tc.TYPE_NAMES.index(name)


def test_closed_forms():
    n = 1000
    c = gpu_census(n, [], [])
    assert c[0] == C3(n) and sum(c[1:]) == 0
    m = 120
    s, d = map(list, zip(*[(a, b) for a in range(m) for b in range(m) if a != b]))
    assert gpu_census(m, s, d)[idx("300")] == C3(m)
    s, d = map(list, zip(*[(a, b) for a in range(m) for b in range(m) if a < b]))
    assert gpu_census(m, s, d)[idx("030T")] == C3(m)
    c = gpu_census(n, [0, 1, 2], [1, 2, 0])
    want = [0] * 16
    want[idx("030C")] = 1
    want[idx("012")] = 3 * (n - 3)
    want[0] = C3(n) - 1 - 3 * (n - 3)
    assert c == want


@pytest.mark.parametrize("n", [3, 100, 50_000])
def test_stars(n):
    # the hub task has |N(u)|+|N(v)| = n: at 50k it is split over CTA chunks
    leaves = np.arange(1, n, dtype=np.int32)
    hub = np.zeros(n - 1, dtype=np.int32)
    for name in ("default", "cta"):
        c = gpu_census(n, hub, leaves, opts(name))
        assert c[idx("021D")] == (n - 1) * (n - 2) // 2 and c[0] == C3(n - 1) and sum(c) == C3(n)
        c = gpu_census(n, leaves, hub, opts(name))
        assert c[idx("021U")] == (n - 1) * (n - 2) // 2 and c[0] == C3(n - 1)


def test_large_n_needs_128_bit_null_count():
    n = 5_000_000  # C(n,3) > 2^64
    c = gpu_census(n, [0, 1], [1, 2])
    assert c[0] == C3(n) - c[idx("021C")] - c[idx("012")]
    assert c[0] >= 1 << 64
    assert sum(c) == C3(n)


def test_input_policy():
    base = gpu_census(6, [0, 1, 2], [1, 2, 3])
    assert gpu_census(6, [0, 1, 2, 0, 0, 4], [1, 2, 3, 1, 0, 4]) == base
    assert gpu_census(2, [0], [1]) == [0] * 16
    assert gpu_census(0, [], []) == [0] * 16
    with pytest.raises(tc.TcError) as e:
        gpu_census(3, [0, 1], [1, 3])
    assert e.value.status == tc.TC_ERR_ID_RANGE
    with pytest.raises(tc.TcError) as e:
        gpu_census(3, [0, -1], [1, 2])
    assert e.value.status == tc.TC_ERR_ID_RANGE


def test_build_layout_matches_definition():
    rng = np.random.default_rng(9)
    n = 500
    src, dst = rand_graph(rng, n, 0.02, 0.3)
    src = np.concatenate([src, src[:50], np.arange(10, dtype=np.int32)])  # dups + loops
    dst = np.concatenate([dst, dst[:50], np.arange(10, dtype=np.int32)])
    g = tc.tc_graph_build(n, src, dst)
    try:
        rp, adj = tc.tc_graph_export(g)
        st = tc.tc_graph_stats(g)
    finally:
        tc.tc_graph_free(g)
    arcs = {(int(a), int(b)) for a, b in zip(src, dst) if a != b}
    rows = {x: {} for x in range(n)}
    for a, b in arcs:
        rows[a][b] = rows[a].get(b, 0) | 1
        rows[b][a] = rows[b].get(a, 0) | 2
    for x in range(n):
        got = [(int(e) >> 2, int(e) & 3) for e in adj[rp[x]:rp[x + 1]]]
        assert got == sorted(rows[x].items()), x
    og = oracle.Graph(n, src, dst).stats()
    for k in ("arcs", "dyads", "mutual", "asym", "merged_entries", "max_degree"):
        assert st[k] == og[k], k


def test_build_crowded_hub_rows_match_definition():
    """Hub rows whose neighbour ids crowd into a few id ranges, with many
    duplicate and reversed arcs: the build's long-row path splits a hub row by
    id range, and ranges of more than 512 entries (sorted in shared-memory
    pieces) and of more than 8192 (pieces merged pairwise) take its slower
    forms.  The hubs' rows against the definition, every statistic and the
    census against the oracle."""
    rng = np.random.default_rng(31)
    n = 200_000
    parts = []

    def arcs_to(h, ids, reps):
        t = np.repeat(ids, reps)
        out = rng.random(t.size) < 0.6
        parts.append((np.where(out, h, t), np.where(out, t, h)))

    arcs_to(7, rng.choice(n, 6000, replace=False), rng.integers(1, 3, 6000))  # spread: many short ranges
    arcs_to(11, np.arange(100, 400), 40)                             # one range of ~12k entries
    arcs_to(13, np.arange(2000, 2101), 30)                           # two ranges of 1.4-1.6k entries
    parts.append((rng.integers(0, n, 150_000), rng.integers(0, n, 150_000)))
    src = np.concatenate([p[0] for p in parts]).astype(np.int32)
    dst = np.concatenate([p[1] for p in parts]).astype(np.int32)
    g = tc.tc_graph_build(n, src, dst)
    try:
        rp, adj = tc.tc_graph_export(g)
        st = tc.tc_graph_stats(g)
        got = tc.tc_census(g)
    finally:
        tc.tc_graph_free(g)
    for h in (7, 11, 13):
        row = {}
        for a, b in zip(src.tolist(), dst.tolist()):
            if a == b:
                continue
            if a == h:
                row[b] = row.get(b, 0) | 1
            elif b == h:
                row[a] = row.get(a, 0) | 2
        got_row = [(int(e) >> 2, int(e) & 3) for e in adj[rp[h]:rp[h + 1]]]
        assert got_row == sorted(row.items()), h
    og = oracle.Graph(n, src, dst)
    try:
        ost = og.stats()
        want = og.census(THREADS)
    finally:
        og.close()
    for k in ("arcs", "dyads", "mutual", "asym", "merged_entries", "max_degree"):
        assert st[k] == ost[k], k
    assert got == want


def csr_definition(n, src, dst, undirected=False):
    """The tagged combined CRS by its definition (numpy): every arc x->y, not
    a self-loop, gives neighbour y of row x with tag bit 0 and neighbour x of
    row y with tag bit 1 (both bits for an undirected edge); one word per
    (row, neighbour), tags OR-ed, rows sorted by neighbour."""
    s = np.asarray(src, dtype=np.int64)
    d = np.asarray(dst, dtype=np.int64)
    keep = s != d
    s, d = s[keep], d[keep]
    t_out, t_in = (3, 3) if undirected else (1, 2)
    rows = np.concatenate([s, d])
    nbr = np.concatenate([d, s])
    tag = np.concatenate([np.full(s.size, t_out), np.full(s.size, t_in)]).astype(np.int64)
    uk, inv = np.unique(rows * n + nbr, return_inverse=True)
    t = np.zeros(uk.size, dtype=np.int64)
    np.bitwise_or.at(t, inv, tag)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, uk // n + 1, 1)
    return np.cumsum(rp), ((uk % n) << 2 | t).astype(np.uint32)


def hub_mix(rng, n, m0, hubs):
    """Random arcs plus, for each (hub, entries), that many arcs between the
    hub and random vertices in either direction, a third of them repeated."""
    parts = [(rng.integers(0, n, m0), rng.integers(0, n, m0))]
    for h, L in hubs:
        other = rng.integers(0, n, L)
        other = np.concatenate([other, other[: L // 3]])
        out = rng.random(other.size) < 0.5
        parts.append((np.where(out, h, other), np.where(out, other, h)))
    loops = rng.integers(0, n, 100)
    parts.append((loops, loops))
    src = np.concatenate([p[0] for p in parts]).astype(np.int32)
    dst = np.concatenate([p[1] for p in parts]).astype(np.int32)
    perm = rng.permutation(src.size)
    return src[perm], dst[perm]


@pytest.mark.parametrize("undirected", [False, True])
def test_build_rows_of_every_length_match_definition(undirected):
    """Whole-graph layout against the definition, rows of every length: short
    rows, rows of 513-4000 entries inside buckets that fit in shared memory
    (sorted and merged in the bucket), and hub rows whose buckets do not fit
    (the long-row path); duplicates, reversed arcs and self-loops."""
    rng = np.random.default_rng(41)
    n = 65536
    hubs = [(1000 * i + 7, int(rng.integers(513, 4000))) for i in range(40)] + [(50_021, 12_000), (60_013, 30_000)]
    src, dst = hub_mix(rng, n, 200_000, hubs)
    g = tc.tc_graph_build(n, src, dst, undirected=undirected)
    try:
        rp, adj = tc.tc_graph_export(g)
        st = tc.tc_graph_stats(g)
    finally:
        tc.tc_graph_free(g)
    want_rp, want_adj = csr_definition(n, src, dst, undirected)
    assert np.array_equal(rp, want_rp)
    assert np.array_equal(adj, want_adj)
    deg = np.diff(want_rp)
    assert st["merged_entries"] == int((deg.astype(np.int64) ** 2).sum())
    assert st["max_degree"] == int(deg.max())


def test_build_batched_rows_match_definition():
    """A batch whose buckets span graph boundaries: every graph's layout
    against the definition (local ids, the split point of each row counted
    against the row's local id through the census)."""
    rng = np.random.default_rng(43)
    ns = [5000, 7001, 3000, 1]
    graphs = [hub_mix(rng, n, 6 * n, [(n // 2, 700)] if n > 1000 else []) if n > 1 else
              (np.zeros(0, np.int32), np.zeros(0, np.int32)) for n in ns]
    off = np.cumsum([0] + [s.size for s, _ in graphs])
    src = np.concatenate([s for s, _ in graphs]).astype(np.int32)
    dst = np.concatenate([d for _, d in graphs]).astype(np.int32)
    hs = tc.tc_graph_build_batched(ns, off, src, dst)
    try:
        for h, n, (s, d) in zip(hs, ns, graphs):
            rp, adj = tc.tc_graph_export(h)
            want_rp, want_adj = csr_definition(n, s, d)
            assert np.array_equal(rp, want_rp)
            assert np.array_equal(adj, want_adj)
            if n > 1:
                assert tc.tc_census(h) == oracle.census(n, s, d)
    finally:
        for h in hs:
            tc.tc_graph_free(h)


def test_device_inputs_and_device_output_on_a_stream():
    import torch
    a = synth.c1()
    gold = json.load(open(os.path.join(GOLDEN, "census_c1.json")))["census"]
    s = torch.cuda.Stream()
    src = torch.from_numpy(a.src).cuda()
    dst = torch.from_numpy(a.dst).cuda()
    torch.cuda.synchronize()
    g = tc.tc_graph_build(a.n, src, dst, stream=s)
    try:
        out = torch.zeros(17, dtype=torch.int64, device="cuda")
        tc.tc_census(g, None, out=out, stream=s)
        s.synchronize()
        assert tc.census_from_device_words(out.cpu().tolist()) == gold
    finally:
        tc.tc_graph_free(g)


def test_repeated_calls_are_identical():
    rng = np.random.default_rng(77)
    src, dst = hub_graph(rng, 5000, 2, 3000, 20000, 0.3)
    g = tc.tc_graph_build(5000, src, dst)
    try:
        first = tc.tc_census(g)
        for _ in range(5):
            assert tc.tc_census(g) == first
    finally:
        tc.tc_graph_free(g)


def test_batch_plan_replays_match_oracle():
    import torch
    rng = np.random.default_rng(123)
    arcs, ns = [], []
    for k in range(40):
        n = int(rng.integers(3, 300))
        if k % 7 == 0:
            s_, d_ = hub_graph(rng, max(n, 2600), 1, 2500, 2000, 0.2)
            n = max(n, 2600)
        else:
            s_, d_ = rand_graph(rng, n, float(rng.choice([0.01, 0.05, 0.2])), 0.3)
        arcs.append((s_, d_))
        ns.append(n)
    off = np.cumsum([0] + [a[0].size for a in arcs])
    src = np.concatenate([a[0] for a in arcs]).astype(np.int32)
    dst = np.concatenate([a[1] for a in arcs]).astype(np.int32)
    want = [oracle.census(n, a[0], a[1], threads=THREADS) for n, a in zip(ns, arcs)]
    gs = tc.tc_graph_build_batched(ns, off, src, dst)
    try:
        for name in ("default", "fwd_map_all", "fwd_search_all", "persistent", "persistent_small"):
            out = torch.zeros(17 * len(gs), dtype=torch.int64, device="cuda")
            plan = tc.tc_plan_create(gs, out, opts(name))
            try:
                for _ in range(2):
                    out.zero_()
                    tc.tc_plan_run(plan)
                    torch.cuda.synchronize()
                    words = out.cpu().tolist()
                    got = [tc.census_from_device_words(words[17 * i:17 * i + 17]) for i in range(len(gs))]
                    assert got == want, name
            finally:
                tc.tc_plan_free(plan)
        # a plan over a reordered subset writes results in its own order
        pick = [5, 0, 33, 7]
        out = torch.zeros(17 * len(pick), dtype=torch.int64, device="cuda")
        plan = tc.tc_plan_create([gs[i] for i in pick], out)
        tc.tc_plan_run(plan)
        torch.cuda.synchronize()
        words = out.cpu().tolist()
        tc.tc_plan_free(plan)
        assert [tc.census_from_device_words(words[17 * i:17 * i + 17]) for i in range(4)] == [want[i] for i in pick]
    finally:
        for g in gs:
            tc.tc_graph_free(g)


def test_autotune_returns_valid_options_and_same_counts(tmp_path):
    rng = np.random.default_rng(8)
    src, dst = hub_graph(rng, 4000, 2, 2000, 15000, 0.3)
    want = oracle.census(4000, src, dst, threads=THREADS)
    g = tc.tc_graph_build(4000, src, dst)
    try:
        best, ms, trials = tc.tc_autotune([g], max_trials=12)
        assert 1 <= trials <= 12 and ms > 0
        assert 0 <= best.thr_thread <= best.thr_warp and 256 <= best.chunk <= 1024
        assert tc.tc_census(g, best) == want
        cache = tmp_path / "tune.json"
        o1 = tc.autotune([g], cache_path=str(cache), max_trials=6)
        o2 = tc.autotune([g], cache_path=str(cache), max_trials=6)  # served from the cache
        assert [getattr(o1, k) for k in tc.TUNED_FIELDS] == [getattr(o2, k) for k in tc.TUNED_FIELDS]
        assert tc.tc_census(g, o2) == want
    finally:
        tc.tc_graph_free(g)


# ------------------------------------------------------------ forward path

@pytest.mark.parametrize("seed", range(4))
def test_forward_path_finds_each_triangle_once(seed):
    """Every triangle is found exactly once, whichever lookup form its owner
    takes (tag map, search, or a mix), and the lookups equal the list
    lengths the ranking defines (computed here with numpy)."""
    rng = np.random.default_rng(300 + seed)
    n = 20_000
    src, dst = hub_graph(rng, n, hubs=4, hub_deg=int(rng.integers(1000, 6000)), extra=80_000, recip=0.3)
    want = oracle.census(n, src, dst, threads=THREADS)
    s = src.astype(np.int64)
    d = dst.astype(np.int64)
    keep = s != d
    pair = np.unique(np.minimum(s[keep], d[keep]) * n + np.maximum(s[keep], d[keep]))
    u, v = pair // n, pair % n
    deg = np.bincount(u, minlength=n) + np.bincount(v, minlength=n)
    cls = np.where(deg > 0, np.floor(np.log2(np.maximum(deg, 1))), 0).astype(np.int64)
    rk = cls * n + np.arange(n)  # the rank order: (floor(log2 d), id)
    lo = np.where(rk[u] < rk[v], u, v)
    hi = np.where(rk[u] < rk[v], v, u)
    nplus = np.bincount(lo, minlength=n)
    order = np.lexsort((rk[hi], lo))
    start = np.concatenate([[0], np.cumsum(nplus)])
    pos = np.arange(order.size) - start[lo[order]]
    suffix = nplus[lo[order]] - pos - 1
    # a forward list of at most 16 entries is looked up whole (its entries
    # ranked below the owner cannot be hits)
    looked = np.where(nplus[lo[order]] <= 16, nplus[lo[order]], suffix)
    owner_has_fwd = nplus[hi[order]] > 0
    lookups = int(looked[owner_has_fwd].sum())
    for name in ("fwd", "fwd_map_all", "fwd_search_all", "fwd_map_mid", "fwd_row_tasks"):
        c, p = forward_profile(n, src, dst, name)
        assert c == want, name
        assert p["map_triangles"] + p["search_triangles"] == triangles(want), name
        assert p["map_lookups"] + p["search_lookups"] == lookups, name
        assert p["fwd_entries"] == pair.size, name
    _, p = forward_profile(n, src, dst, "fwd_search_all")
    assert p["map_lookups"] == 0 and p["map_items"] == 0


# ------------------------------------------------------- exact-cost binning

def union_sizes(n, src, dst):
    """|S| = |N(u) u N(v) \\ {u, v}| of every canonical dyad u < v, from a
    sparse adjacency product (c_uv = common neighbours)."""
    import scipy.sparse as sp
    s = src.astype(np.int64)
    d = dst.astype(np.int64)
    keep = s != d
    pair = np.unique(np.minimum(s[keep], d[keep]) * n + np.maximum(s[keep], d[keep]))
    u, v = pair // n, pair % n
    A = sp.coo_matrix((np.ones(u.size, np.int64), (u, v)), shape=(n, n)).tocsr()
    A = ((A + A.T) > 0).astype(np.int64)
    deg = np.asarray(A.sum(axis=1)).ravel()
    common = np.asarray((A @ A)[u, v]).ravel()
    return u, v, deg, deg[u] + deg[v] - 2 - common


@pytest.mark.parametrize("seed", range(2))
def test_exact_binning_bins_by_union_size(seed):
    """bin_mode = TC_BIN_EXACT puts a merge task in the thread bin when
    |S| + 2 <= thr_thread and in the warp bin when <= thr_warp: the bin
    counts equal those |S| gives (computed here from the adjacency), differ
    from the degree-sum rule's, and the counts equal the oracle's."""
    rng = np.random.default_rng(900 + seed)
    n = 600
    src, dst = rand_graph(rng, n, 0.06, 0.3)
    want = oracle.census(n, src, dst, threads=THREADS)
    u, v, deg, S = union_sizes(n, src, dst)
    T, W = int(np.percentile(S + 2, 40)), int(np.percentile(S + 2, 80))  # thresholds inside the spread
    got = {}
    for mode, cost in ((tc.TC_BIN_EXACT, S + 2), (tc.TC_BIN_HEURISTIC, deg[u] + deg[v])):
        o = tc.tc_opts_default(tri_path=MERGE, bin_mode=mode, own_min=0, thr_thread=T, thr_warp=W, profile=1)
        g = tc.tc_graph_build(n, src, dst)
        try:
            assert tc.tc_census(g, o) == want, mode
            p = tc.tc_census_profile()
        finally:
            tc.tc_graph_free(g)
        b = p["bin_tasks"]
        assert b[0] == int((cost <= T).sum()), mode
        assert b[1] == int(((cost > T) & (cost <= W)).sum()), mode
        assert b[2] + b[3] == int((cost > W).sum()), mode
        assert (p["ms_exact_cost"] > 0) == (mode == tc.TC_BIN_EXACT)
        got[mode] = b
    assert got[tc.TC_BIN_EXACT] != got[tc.TC_BIN_HEURISTIC]


# ------------------------------------------------------------ path routing

def mixed_batch(rng, k):
    """Near-regular random graphs and hub graphs, alternating."""
    arcs, ns = [], []
    for i in range(k):
        if i % 2:
            n = int(rng.integers(2000, 6000))
            s_, d_ = hub_graph(rng, n, 2, int(rng.integers(500, 1500)), 4 * n, 0.2)
        else:
            n = int(rng.integers(100, 400))
            s_, d_ = rand_graph(rng, n, float(rng.choice([0.02, 0.05])), 0.3)
        arcs.append((s_, d_))
        ns.append(n)
    off = np.cumsum([0] + [a[0].size for a in arcs])
    return ns, off, np.concatenate([a[0] for a in arcs]).astype(np.int32), \
        np.concatenate([a[1] for a in arcs]).astype(np.int32), arcs


def test_auto_routing_never_changes_counts():
    """Whatever path the router gives each graph (the degree-skew rule, or
    models that send every graph one way, or a random one), the batched
    census, its plan and its 64-code form equal the oracle's."""
    import torch
    from oracle import mlp as omlp
    rng = np.random.default_rng(404)
    ns, off, src, dst, arcs = mixed_batch(rng, 12)
    want = [oracle.census(n, a[0], a[1], threads=THREADS) for n, a in zip(ns, arcs)]
    gs = tc.tc_graph_build_batched(ns, off, src, dst)
    try:
        feat = tc.tc_path_features(gs)
        rule = [tc.TC_TRI_MERGE if f[4] * 8.0 < 3.0 else tc.TC_TRI_FORWARD for f in feat]
        assert tc.tc_path_route(gs) == rule
        assert set(rule) == {tc.TC_TRI_FORWARD, tc.TC_TRI_MERGE}  # both paths in one census
        models = []
        for bias in ([0.0, 50.0, 0.0, 0.0], [50.0, 0.0, 0.0, 0.0], None):
            p = omlp.init(7).astype(np.float32)
            if bias is not None:
                p[-4:] = bias  # outputs: log2 time forward, merge
            models.append((bias, p))
        for bias, p in [(None, None)] + models:
            tc.tc_path_model_load(p)
            if bias == [0.0, 50.0, 0.0, 0.0]:
                assert tc.tc_path_route(gs) == [tc.TC_TRI_FORWARD] * len(gs)
            if bias == [50.0, 0.0, 0.0, 0.0]:
                assert tc.tc_path_route(gs) == [tc.TC_TRI_MERGE] * len(gs)
            o = tc.tc_opts_default(tri_path=tc.TC_TRI_AUTO)
            assert tc.tc_census_batched(gs, o) == want
            codes = tc.tc_census_codes_batched(gs, o)
            assert [fold(c) for c in codes] == want
            out = torch.zeros(17 * len(gs), dtype=torch.int64, device="cuda")
            plan = tc.tc_plan_create(gs, out, o)
            tc.tc_plan_run(plan)
            torch.cuda.synchronize()
            tc.tc_plan_free(plan)
            words = out.cpu().tolist()
            assert [tc.census_from_device_words(words[17 * i:17 * i + 17]) for i in range(len(gs))] == want
    finally:
        tc.tc_path_model_load(None)
        for g in gs:
            tc.tc_graph_free(g)
