"""Pins for the CPU oracle (no GPU).

The oracle is trusted only because these tests tie it to things other than
itself: the exhaustive three- and four-vertex cases, the O(n^3) definition,
closed forms, invariants of the census, an external black-box census routine
and the textbook G(n,p) expectation.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth

NAMES = oracle.TYPE_NAMES
ORBIT = [1, 6, 3, 3, 3, 6, 6, 6, 6, 2, 3, 3, 3, 6, 6, 1]

# bit of e(a,b) in the 6-bit code, vertices 0=u 1=v 2=w (Fig. "Triad Code Algorithm")
BIT = {(0, 1): 1, (1, 0): 2, (0, 2): 4, (2, 0): 8, (1, 2): 16, (2, 1): 32}


def code_arcs(c):
    return [ab for ab, bit in BIT.items() if c & bit]


def arcs_code(arcs):
    return sum(BIT[ab] for ab in arcs)


def man_digits(c):
    arcs = set(code_arcs(c))
    m = a = 0
    for x, y in ((0, 1), (0, 2), (1, 2)):
        f, b = (x, y) in arcs, (y, x) in arcs
        m += f and b
        a += f != b
    return m, a, 3 - m - a


def nx_census(n, src, dst):
    nx = pytest.importorskip("networkx")
    G = nx.DiGraph()
    G.add_nodes_from(range(n))
    G.add_edges_from((int(s), int(d)) for s, d in zip(src, dst) if s != d)
    tc = nx.triadic_census(G)
    return [tc[name] for name in NAMES]


# ----------------------------------------------------------------- n = 3

def test_table_man_digits_orbits_and_invariance():
    T = oracle.triad_table()
    for c in range(64):
        m, a, n0 = man_digits(c)
        assert NAMES[T[c]][:3] == f"{m}{a}{n0}", c
    # S3 invariance: relabelling the three vertices keeps the type
    for c in range(64):
        arcs = code_arcs(c)
        for perm in itertools.permutations(range(3)):
            pc = arcs_code([(perm[x], perm[y]) for x, y in arcs])
            assert T[pc] == T[c]
    # orbit sizes of the 16 classes (64 labelled triads in total)
    sizes = [sum(1 for c in range(64) if T[c] == t) for t in range(16)]
    assert sizes == ORBIT


def test_table_matches_external_routine():
    T = oracle.triad_table()
    for c in range(64):
        arcs = code_arcs(c)
        src = [a for a, _ in arcs]
        dst = [b for _, b in arcs]
        ref = nx_census(3, src, dst)
        assert ref[T[c]] == 1 and sum(ref) == 1, c


def test_all_64_triads_one_count_each():
    T = oracle.triad_table()
    for c in range(64):
        arcs = code_arcs(c)
        src = np.array([a for a, _ in arcs], dtype=np.int32)
        dst = np.array([b for _, b in arcs], dtype=np.int32)
        want = [0] * 16
        want[T[c]] = 1
        assert oracle.brute_census(3, src, dst) == want
        assert oracle.census(3, src, dst) == want


# ----------------------------------------------------------------- n = 4

def test_all_4096_four_vertex_digraphs():
    pairs = [(a, b) for a in range(4) for b in range(4) if a != b]
    for mask in range(1 << 12):
        arcs = [pairs[k] for k in range(12) if mask >> k & 1]
        src = np.array([a for a, _ in arcs], dtype=np.int32)
        dst = np.array([b for _, b in arcs], dtype=np.int32)
        b = oracle.brute_census(4, src, dst)
        assert oracle.census(4, src, dst) == b, mask
        assert sum(b) == 4


def test_four_vertex_sample_vs_external():
    pairs = [(a, b) for a in range(4) for b in range(4) if a != b]
    rng = np.random.default_rng(7)
    for mask in rng.integers(0, 1 << 12, size=300):
        arcs = [pairs[k] for k in range(12) if int(mask) >> k & 1]
        src = [a for a, _ in arcs]
        dst = [b for _, b in arcs]
        assert oracle.census(4, src, dst) == nx_census(4, src, dst)


# ----------------------------------------------------------------- random

def rand_graph(rng, n, p, r):
    s, d = np.nonzero(rng.random((n, n)) < p)
    keep = s != d
    s, d = s[keep], d[keep]
    rec = rng.random(s.size) < r
    src = np.concatenate([s, d[rec]]).astype(np.int32)
    dst = np.concatenate([d, s[rec]]).astype(np.int32)
    return src, dst


@pytest.mark.parametrize("seed", range(12))
def test_random_graphs_vs_brute(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 90))
    p = float(rng.choice([0.01, 0.05, 0.2, 0.5, 0.9]))
    r = float(rng.choice([0.0, 0.3, 1.0]))
    src, dst = rand_graph(rng, n, p, r)
    b = oracle.brute_census(n, src, dst)
    assert oracle.census(n, src, dst, threads=1) == b
    assert oracle.census(n, src, dst, threads=4) == b
    assert sum(b) == oracle.choose3(n)


@pytest.mark.parametrize("seed", range(8))
def test_common_neighbour_sums_follow_closed_triads(seed):
    # The CUDA path drops shared elements below both endpoints of a dyad and
    # restores their dyadic share from the final counts: summed over the
    # asymmetric (mutual) dyads, |N(u) n N(v)| equals the number of closed
    # triads weighted by how many asymmetric (mutual) dyads each has.  Checked
    # here by brute force on the oracle's adjacency and brute-force census.
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(4, 70))
    src, dst = rand_graph(rng, n, float(rng.choice([0.05, 0.2, 0.6])), float(rng.choice([0.0, 0.3, 1.0])))
    g = oracle.Graph(n, src, dst)
    arcs = set(zip(src.tolist(), dst.tolist())) - {(i, i) for i in range(n)}
    asym = mutual = 0
    for u in range(n):
        for v in range(u + 1, n):
            a, b = (u, v) in arcs, (v, u) in arcs
            if a or b:
                c = g.common(u, v)
                if a and b:
                    mutual += c
                else:
                    asym += c
    t = dict(zip(NAMES, oracle.brute_census(n, src, dst)))
    c120 = t["120D"] + t["120U"] + t["120C"]
    assert asym == 3 * (t["030T"] + t["030C"]) + 2 * c120 + t["210"]
    assert mutual == c120 + 2 * t["210"] + 3 * t["300"]


@pytest.mark.parametrize("seed", range(4))
def test_random_graphs_vs_external(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(5, 50))
    src, dst = rand_graph(rng, n, 0.15, 0.3)
    assert oracle.census(n, src, dst) == nx_census(n, src, dst)


# ----------------------------------------------------------------- closed forms

def C3(n):
    return n * (n - 1) * (n - 2) // 6


def idx(name):
    return NAMES.index(name)


@pytest.mark.parametrize("n", [3, 10, 57])
def test_closed_forms(n):
    # empty graph: every triad null
    c = oracle.census(n, [], [])
    assert c[0] == C3(n) and sum(c[1:]) == 0
    # complete mutual graph: every triad 300
    s, d = zip(*[(a, b) for a in range(n) for b in range(n) if a != b])
    c = oracle.census(n, s, d)
    assert c[idx("300")] == C3(n) and sum(c) == C3(n)
    # transitive tournament a->b for a<b: every triad 030T
    s, d = zip(*[(a, b) for a in range(n) for b in range(n) if a < b])
    c = oracle.census(n, s, d)
    assert c[idx("030T")] == C3(n)
    # lone directed 3-cycle
    c = oracle.census(n, [0, 1, 2], [1, 2, 0])
    want = [0] * 16
    want[idx("030C")] = 1
    want[idx("012")] = 3 * (n - 3)
    want[0] = C3(n) - 1 - 3 * (n - 3)
    assert c == want
    # out-star and in-star from vertex 0
    leaves = list(range(1, n))
    c = oracle.census(n, [0] * (n - 1), leaves)
    assert c[idx("021D")] == (n - 1) * (n - 2) // 2 and c[0] == C3(n - 1)
    assert sum(c) == C3(n)
    c = oracle.census(n, leaves, [0] * (n - 1))
    assert c[idx("021U")] == (n - 1) * (n - 2) // 2 and c[0] == C3(n - 1)


def test_input_policy():
    # self-loops dropped, duplicate arcs collapse, isolated vertices count
    base = oracle.census(6, [0, 1, 2], [1, 2, 3])
    assert oracle.census(6, [0, 1, 2, 0, 0, 4], [1, 2, 3, 1, 0, 4]) == base
    assert oracle.census(2, [0], [1]) == [0] * 16
    assert oracle.census(0, [], []) == [0] * 16
    with pytest.raises(ValueError):
        oracle.Graph(3, [0], [3])


# ----------------------------------------------------------------- invariants

# (M, A, N) of each type from its MAN name
MAN = [tuple(int(ch) for ch in nm[:3]) for nm in NAMES]


def check_invariants(n, src, dst, c):
    g = oracle.Graph(n, src, dst)
    st = g.stats()
    assert sum(c) == C3(n)
    # each dyad lies in n-2 triads
    M, A = st["mutual"], st["asym"]
    N0 = n * (n - 1) // 2 - M - A
    assert sum(MAN[t][0] * c[t] for t in range(16)) == M * (n - 2)
    assert sum(MAN[t][1] * c[t] for t in range(16)) == A * (n - 2)
    assert sum(MAN[t][2] * c[t] for t in range(16)) == N0 * (n - 2)


def transpose_swap(c):
    out = list(c)
    for a, b in (("021D", "021U"), ("111D", "111U"), ("120D", "120U")):
        out[idx(a)], out[idx(b)] = c[idx(b)], c[idx(a)]
    return out


@pytest.mark.parametrize("seed", range(3))
def test_invariants_relabel_transpose(seed):
    rng = np.random.default_rng(1000 + seed)
    n = 300
    src, dst = rand_graph(rng, n, 0.03, 0.4)
    c = oracle.census(n, src, dst)
    check_invariants(n, src, dst, c)
    pi = rng.permutation(n).astype(np.int32)
    assert oracle.census(n, pi[src], pi[dst]) == c
    assert oracle.census(n, dst, src) == transpose_swap(c)


def test_oriented_dag_has_no_mutual_or_cyclic_types():
    a = synth.rmat(10, 4, orient_down=True, permute=True, seed=11)
    c = oracle.census(a.n, a.src, a.dst)
    for name in ("102", "111D", "111U", "030C", "201", "120D", "120U", "120C", "210", "300"):
        assert c[idx(name)] == 0, name
    check_invariants(a.n, a.src, a.dst, c)


# ----------------------------------------------------------------- G(n,p)

def gnp_expectation(n, p, r):
    """Textbook expected census of a graph whose dyads are independent:
    mutual pm, asymmetric pa per direction, null p0."""
    pm = p * p + 2 * p * (1 - p) * r
    pa = p * (1 - p) * (1 - r)
    p0 = (1 - p) ** 2
    per = {
        "003": p0 ** 3, "012": 6 * pa * p0 ** 2, "102": 3 * pm * p0 ** 2,
        "021D": 3 * pa ** 2 * p0, "021U": 3 * pa ** 2 * p0, "021C": 6 * pa ** 2 * p0,
        "111D": 6 * pm * pa * p0, "111U": 6 * pm * pa * p0,
        "030T": 6 * pa ** 3, "030C": 2 * pa ** 3, "201": 3 * pm ** 2 * p0,
        "120D": 3 * pm * pa ** 2, "120U": 3 * pm * pa ** 2, "120C": 6 * pm * pa ** 2,
        "210": 6 * pm ** 2 * pa, "300": pm ** 3,
    }
    assert abs(sum(per.values()) - 1) < 1e-12
    return [C3(n) * per[nm] for nm in NAMES]


def test_gnp_counts_match_expectation():
    a = synth.c1()
    c = oracle.census(a.n, a.src, a.dst)
    exp = gnp_expectation(1024, 8 / 1023, 0.25)
    for t in range(16):
        tol = 18 * math.sqrt(exp[t]) + 0.02 * exp[t] + 5
        assert abs(c[t] - exp[t]) <= tol, (NAMES[t], c[t], exp[t])
    check_invariants(a.n, a.src, a.dst, c)


# ------------------------------------------------------ 64-code census (f1)

def fold(codes):
    T = oracle.triad_table()
    out = [0] * 16
    for c, k in enumerate(codes):
        out[T[c]] += k
    return out


def one_hot(n, **codes):
    out = [0] * 64
    for c, k in codes.items():
        out[int(c[1:])] = k
    return out


def test_codes_hand_cases():
    # worked by hand from Fig. "Triad Code Algorithm" and the canonical test
    cases = [
        # path 0->1->2: <0,1> with w = 2 > v counts it: 1 + 16 e(1,2) = 17
        (3, [(0, 1), (1, 2)], dict(c17=1)),
        # single arc: the dyadic term of <1,2>, code pre
        (3, [(1, 2)], dict(c1=1)),
        (3, [(2, 1)], dict(c2=1)),
        (3, [(0, 1), (1, 0)], dict(c3=1)),
        # transitive triangle: <0,1> with w = 2: 1 + 4 e(0,2) + 16 e(1,2) = 21
        (3, [(0, 1), (1, 2), (0, 2)], dict(c21=1)),
        # 0->2->1: <0,2> with w = 1 (0 < 1 < 2, 1 not a neighbour of 0):
        # pre 1 + 16 e(2,1) = 17; <1,2> with w = 0 < u does not count
        (3, [(0, 2), (2, 1)], dict(c17=1)),
        # one arc among four vertices: two dyadic triads, two null ones
        (4, [(0, 1)], dict(c0=2, c1=2)),
    ]
    for n, arcs, want in cases:
        src = np.array([a for a, _ in arcs], dtype=np.int32)
        dst = np.array([b for _, b in arcs], dtype=np.int32)
        got = oracle.brute_census_codes(n, src, dst)
        assert got == one_hot(n, **want), (arcs, [i for i, k in enumerate(got) if k])
        assert oracle.census_codes(n, src, dst) == got


def test_codes_all_64_triads_and_4096_four_vertex_digraphs():
    for c in range(64):
        arcs = code_arcs(c)
        src = np.array([a for a, _ in arcs], dtype=np.int32)
        dst = np.array([b for _, b in arcs], dtype=np.int32)
        b = oracle.brute_census_codes(3, src, dst)
        assert fold(b) == oracle.brute_census(3, src, dst), c
        assert oracle.census_codes(3, src, dst) == b, c
    pairs = [(a, b) for a in range(4) for b in range(4) if a != b]
    for mask in range(1 << 12):
        arcs = [pairs[k] for k in range(12) if mask >> k & 1]
        src = np.array([a for a, _ in arcs], dtype=np.int32)
        dst = np.array([b for _, b in arcs], dtype=np.int32)
        b = oracle.brute_census_codes(4, src, dst)
        assert fold(b) == oracle.brute_census(4, src, dst), mask
        assert oracle.census_codes(4, src, dst) == b, mask


@pytest.mark.parametrize("seed", range(4))
def test_codes_random_graphs_vs_brute(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(10, 40))
    s, d = np.nonzero(rng.random((n, n)) < rng.uniform(0.05, 0.4))
    b = oracle.brute_census_codes(n, s, d)
    assert oracle.census_codes(n, s, d) == b
    assert fold(b) == oracle.census(n, s, d)
    assert sum(b) == math.comb(n, 3)


# -------------------------------------------------------- graph statistics
def numpy_stats(n, src, dst):
    """The statistics from their definitions, by numpy set operations on the
    raw arcs (independent of the oracle's CRS): distinct arcs without loops,
    unordered adjacent pairs, mutual pairs, degrees by bincount over the
    distinct pairs, merged entries = sum over pairs of d_u + d_v."""
    s = np.asarray(src, np.int64)
    d = np.asarray(dst, np.int64)
    keep = s != d
    s, d = s[keep], d[keep]
    arcs = np.unique(s * n + d)
    lo, hi = np.minimum(arcs // n, arcs % n), np.maximum(arcs // n, arcs % n)
    pair, times = np.unique(lo * n + hi, return_counts=True)
    u, v = pair // n, pair % n
    deg = np.bincount(u, minlength=n) + np.bincount(v, minlength=n)
    return {"n": n, "arcs": int(arcs.size), "dyads": int(pair.size), "mutual": int((times == 2).sum()),
            "asym": int((times == 1).sum()), "merged_entries": int((deg[u] + deg[v]).sum()),
            "max_degree": int(deg.max()) if n else 0}


@pytest.mark.parametrize("case", ["c1", "multi", "star", "rmat"])
def test_graph_stats_follow_their_definitions(case):
    """oracle_graph_stats is the reference for the library's statistics and
    for every bench rate (merged entries = sum_v d_v^2, max degree)."""
    rng = np.random.default_rng(7)
    if case == "c1":
        a = synth.c1()
        n, src, dst = a.n, a.src, a.dst
    elif case == "multi":  # duplicates, loops and both directions of some pairs
        n = 300
        src = rng.integers(0, n, 4000)
        dst = rng.integers(0, n, 4000)
        src = np.concatenate([src, dst[:500], np.arange(20)])
        dst = np.concatenate([dst, src[:500], np.arange(20)])
    elif case == "star":  # one hub: max degree n-1, merged entries (n-1)(n-1+1)
        n = 500
        src = np.zeros(n - 1, np.int64)
        dst = np.arange(1, n)
    else:
        a = synth.rmat(12, 8, recip=0.2, seed=9)
        n, src, dst = a.n, a.src, a.dst
    st = oracle.Graph(n, src, dst).stats()
    want = numpy_stats(n, src, dst)
    assert st == want
    if case == "star":
        assert st["max_degree"] == n - 1 and st["merged_entries"] == (n - 1) * n
    # merged entries = sum_v d_v^2 (each vertex's degree counted once per incident pair)
    s = np.asarray(src, np.int64)
    d = np.asarray(dst, np.int64)
    keep = s != d
    pair = np.unique(np.minimum(s[keep], d[keep]) * n + np.maximum(s[keep], d[keep]))
    deg_sq = np.bincount(np.concatenate([pair // n, pair % n]), minlength=n).astype(np.int64) ** 2
    assert st["merged_entries"] == int(deg_sq.sum())
