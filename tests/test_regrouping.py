"""The regroupings the CUDA path uses, checked on the CPU against the method's
definition (Sec. 2.2, Fig. "Subquadratic Triad Census Algorithm") on small
random digraphs, in plain Python.  They involve no kernel; they pin the
identities the kernels rely on:

* per-dyad suffix terms (as if no element were shared) plus the shared-element
  corrections, each triangle corrected once by its lowest dyad (four updates),
  give the per-code counts of the canonical test exactly;
* the dyadic counts split by pre = e(u,v) + 2e(v,u) follow from the sums
  n - d_u - d_v and the closed codes (a closed triad is counted with u < v < w,
  so its canonical dyads have pre values pre, t_u(w), t_v(w))."""
import numpy as np
import pytest

import oracle


def digraph(seed, n, p):
    rng = np.random.default_rng(seed)
    arcs = {(a, b) for a in range(n) for b in range(n) if a != b and rng.random() < p}
    e = lambda a, b: 1 if (a, b) in arcs else 0
    tag = lambda x, w: e(x, w) + 2 * e(w, x)
    nb = {x: sorted(w for w in range(n) if w != x and tag(x, w)) for x in range(n)}
    src = np.array([a for a, _ in arcs], dtype=np.int32)
    dst = np.array([b for _, b in arcs], dtype=np.int32)
    return tag, nb, src, dst


def swap(t):
    return ((t & 1) << 1) | (t >> 1)


CASES = [(1, 8, 0.3), (2, 12, 0.4), (3, 15, 0.25), (4, 20, 0.5), (5, 10, 0.8), (6, 25, 0.15)]


def regrouped(tag, nb, n, drop=None):
    """Per-code counts from the suffix terms and the once-per-triangle
    corrections; `drop` names one correction to leave out (a planted
    mistake the test must notice)."""
    got = [0] * 64
    for u in range(n):
        for v in nb[u]:
            if v <= u:
                continue
            pre = tag(u, v)
            for w in nb[u]:  # suffix of A after v, as if tag_v(w) = 0
                if w > v:
                    got[pre + 4 * tag(u, w)] += 1
            for w in nb[v]:  # suffix of B after u, as if tag_u(w) = 0
                if w > u and w != v:
                    got[pre + 16 * tag(v, w)] += 1
            for w in set(nb[u]) & set(nb[v]):  # each triangle once, by its lowest dyad
                if w > v:
                    tu, tv = tag(u, w), tag(v, w)
                    if drop != "a":
                        got[pre + 4 * tu] -= 1
                    if drop != "b":
                        got[pre + 16 * tv] -= 1
                    if drop != "joint":
                        got[pre + 4 * tu + 16 * tv] += 1
                    if drop != "middle":
                        got[tu + 16 * swap(tv)] -= 1  # dyad <u,w>, middle vertex v
    return got


def defined(tag, nb, n):
    want = [0] * 64
    for u in range(n):
        for v in nb[u]:
            if v <= u:
                continue
            pre = tag(u, v)
            S = (set(nb[u]) | set(nb[v])) - {u, v}
            for w in S:  # the canonical test and the code, as defined
                if v < w or (u < w < v and w not in nb[u]):
                    want[pre + 4 * tag(u, w) + 16 * tag(v, w)] += 1
    return want


@pytest.mark.parametrize("drop", ["a", "b", "joint", "middle"])
def test_each_correction_is_needed(drop):
    tag, nb, _, _ = digraph(4, 20, 0.5)
    assert regrouped(tag, nb, 20, drop) != defined(tag, nb, 20)


@pytest.mark.parametrize("seed,n,p", CASES)
def test_suffix_terms_plus_triangle_corrections_give_the_codes(seed, n, p):
    tag, nb, _, _ = digraph(seed, n, p)
    assert regrouped(tag, nb, n) == defined(tag, nb, n)


@pytest.mark.parametrize("seed,n,p", CASES)
def test_dyadic_codes_from_degree_sums_and_closed_codes(seed, n, p):
    tag, nb, src, dst = digraph(seed, n, p)
    codes = oracle.census_codes(n, src, dst)
    dsum = [0] * 4   # sum of n - d_u - d_v per pre value
    cuv = [0] * 4    # sum of |N(u) n N(v)| per pre value
    for u in range(n):
        for v in nb[u]:
            if v > u:
                pre = tag(u, v)
                dsum[pre] += n - len(nb[u]) - len(nb[v])
                cuv[pre] += len(set(nb[u]) & set(nb[v]))
    closed = [0] * 4
    for c in range(64):
        pre, tu, tv = c & 3, (c >> 2) & 3, (c >> 4) & 3
        if tu and tv:
            for q in (1, 2, 3):
                closed[q] += codes[c] * ((pre == q) + (tu == q) + (tv == q))
    for q in (1, 2, 3):
        assert closed[q] == cuv[q], q
        assert codes[q] == dsum[q] + cuv[q], q


def rank_order_regrouped(tag, nb, n, pos):
    """Suffix terms in id order, but each triangle's correction taken with
    its vertices in the order `pos` (a < b < c by pos, as the forward path's
    degree ranks): the corrections of the three two-edge triads and the full
    triangle, labelled in that order."""
    got = [0] * 64
    for u in range(n):
        for v in nb[u]:
            if v <= u:
                continue
            pre = tag(u, v)
            for w in nb[u]:
                if w > v:
                    got[pre + 4 * tag(u, w)] += 1
            for w in nb[v]:
                if w > u and w != v:
                    got[pre + 16 * tag(v, w)] += 1
    for u in range(n):
        for v in nb[u]:
            for w in nb[v]:
                if not (u < v < w) or w not in nb[u]:
                    continue
                a, b, c = sorted((u, v, w), key=lambda x: pos[x])
                t_ab, t_ac, t_bc = tag(a, b), tag(a, c), tag(b, c)
                got[t_ab + 4 * t_ac] -= 1
                got[t_ab + 16 * t_bc] -= 1
                got[t_ab + 4 * t_ac + 16 * t_bc] += 1
                got[t_ac + 16 * swap(t_bc)] -= 1
    return got


def fold16(codes):
    T = oracle.triad_table()
    out = [0] * 16
    for c in range(1, 64):
        out[T[c]] += codes[c]
    return out


@pytest.mark.parametrize("seed,n,p", CASES)
def test_triangle_corrections_in_any_vertex_order_give_the_same_types(seed, n, p):
    """By type the correction is symmetric in the triangle's vertices (the
    suffix terms counted it once as each vertex's two-edge triad), so the
    16-type census does not depend on the order the triangles are classified
    in; the 64 labelled codes do, which is why the code census keeps id
    order."""
    tag, nb, _, _ = digraph(seed, n, p)
    want = fold16(defined(tag, nb, n))
    rng = np.random.default_rng(seed)
    differ = False
    for _ in range(3):
        pos = rng.permutation(n)
        got = rank_order_regrouped(tag, nb, n, pos)
        assert fold16(got) == want
        differ |= got != defined(tag, nb, n)
    deg = [len(nb[x]) for x in range(n)]
    degree_rank = sorted(range(n), key=lambda x: (int(np.log2(deg[x])) if deg[x] else 0, x))
    pos = [0] * n
    for r, x in enumerate(degree_rank):
        pos[x] = r
    assert fold16(rank_order_regrouped(tag, nb, n, pos)) == want
    if seed == 4:
        assert differ  # the labelled codes move with the order
