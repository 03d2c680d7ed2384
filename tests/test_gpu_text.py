"""Graph files in the Pajek-style text format (tc_graph_build_text) and the
undirected input mode (TC_UNDIRECTED): the census of the parsed graph
against the oracle's census of the same arcs."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1603_02655_b300 as tc
from paper_1603_02655_b300 import build as tcbuild

pytestmark = pytest.mark.gpu
THREADS = 8


@pytest.fixture(scope="module", autouse=True)
def lib(cuda_ok):
    tcbuild.build()
    return tc.load()


def census_text(text, base=1):
    g = tc.tc_graph_build_text(text, base)
    try:
        return tc.tc_census(g), tc.tc_graph_stats(g)
    finally:
        tc.tc_graph_free(g)


def rand_arcs(rng, n, m):
    return rng.integers(0, n, m).astype(np.int32), rng.integers(0, n, m).astype(np.int32)


def test_arcs_with_labels_weights_comments_crlf():
    rng = np.random.default_rng(1)
    n = 500
    s, d = rand_arcs(rng, n, 4000)
    lines = ["% a comment", f"*Vertices {n}"]
    lines += [f'{i + 1} "v{i + 1}" 0.1 0.2' for i in range(0, n, 7)]  # some labelled vertex lines
    lines += ["", "*Arcs"]
    lines += [f"  {a + 1}\t{b + 1} {rng.random():.3f}" for a, b in zip(s, d)]
    text = "\r\n".join(lines) + "\r\n"
    got, st = census_text(text)
    assert got == oracle.census(n, s, d, threads=THREADS)
    assert st["n"] == n


def test_edges_are_mutual_and_zero_based_ids():
    rng = np.random.default_rng(2)
    n = 300
    s, d = rand_arcs(rng, n, 2000)
    text = f"*vertices {n}\n*EDGES\n" + "\n".join(f"{a} {b}" for a, b in zip(s, d)) + "\n"
    got, _ = census_text(text, base=0)
    want = oracle.census(n, np.concatenate([s, d]), np.concatenate([d, s]), threads=THREADS)
    assert got == want
    # the same through the undirected build flag
    g = tc.tc_graph_build(n, s, d, undirected=True)
    try:
        assert tc.tc_census(g) == want
    finally:
        tc.tc_graph_free(g)


def test_mixed_sections_and_lists():
    rng = np.random.default_rng(3)
    n = 400
    sa, da = rand_arcs(rng, n, 1500)
    se, de = rand_arcs(rng, n, 600)
    src, dst = [sa, se, de], [da, de, se]
    lines = [f"*Vertices {n}", "*Arcs"] + [f"{a + 1} {b + 1}" for a, b in zip(sa, da)]
    lines += ["*Edges"] + [f"{a + 1} {b + 1} 2" for a, b in zip(se, de)]
    lines.append("*Arcslist")
    for a in range(0, n, 5):
        nb = rng.choice(n, size=int(rng.integers(0, 30)), replace=False)
        lines.append(" ".join(str(x + 1) for x in [a, *nb]))
        src.append(np.full(nb.size, a, np.int32))
        dst.append(nb.astype(np.int32))
    lines.append("*Edgeslist")
    for a in range(1, n, 9):
        nb = rng.choice(n, size=int(rng.integers(1, 20)), replace=False)
        lines.append(" ".join(str(x + 1) for x in [a, *nb]))
        src += [np.full(nb.size, a, np.int32), nb.astype(np.int32)]
        dst += [nb.astype(np.int32), np.full(nb.size, a, np.int32)]
    got, _ = census_text("\n".join(lines))  # no final newline
    want = oracle.census(n, np.concatenate(src), np.concatenate(dst), threads=THREADS)
    assert got == want


def test_device_text_input():
    import torch
    n = 64
    text = f"*Vertices {n}\n*Arcs\n" + "\n".join(f"{i + 1} {(i * 7) % n + 1}" for i in range(n)) + "\n"
    t = torch.tensor(list(text.encode()), dtype=torch.uint8, device="cuda")
    g = tc.tc_graph_build_text(t, 1)
    try:
        s = np.arange(n, dtype=np.int32)
        assert tc.tc_census(g) == oracle.census(n, s, (s * 7) % n)
    finally:
        tc.tc_graph_free(g)


@pytest.mark.parametrize("text,status", [
    ("*Arcs\n1 2\n", tc.TC_ERR_ARG),                       # no *Vertices
    ("1 2\n*Vertices 3\n", tc.TC_ERR_ARG),                 # data before a header
    ("*Vertices 3\n*Arcs\n1 x\n", tc.TC_ERR_ARG),          # malformed arc line
    ("*Vertices 3\n*Arcs\n1\n", tc.TC_ERR_ARG),            # one id only
    ("*Vertices 3\n*Vertices 4\n", tc.TC_ERR_ARG),         # two orders
    ("*Vertices 3\n*Matrix\n0 1 0\n", tc.TC_ERR_UNSUPPORTED),
    ("*Vertices 3\n*Arcs\n1 4\n", tc.TC_ERR_ID_RANGE),     # id above n
    ("*Vertices 3\n*Arcs\n0 1\n", tc.TC_ERR_ID_RANGE),     # id 0 with base 1
])
def test_errors(text, status):
    with pytest.raises(tc.TcError) as e:
        tc.tc_graph_build_text(text, 1)
    assert e.value.status == status


def test_tiny_and_empty_inputs():
    # n < 3: every count 0; an order without arcs: all triads null; a section
    # header without lines; the 64-code census agrees
    for text, n in (("*Vertices 0\n", 0), ("*Vertices 2\n*Arcs\n1 2\n", 2), ("*Vertices 5\n*Arcs\n", 5),
                    ("*Vertices 4\n*Edges\n% nothing\n\n", 4)):
        g = tc.tc_graph_build_text(text, 1)
        try:
            want = [0] * 16
            want[0] = n * (n - 1) * (n - 2) // 6 if n >= 3 else 0
            assert tc.tc_census(g) == want, text
            codes = tc.tc_census_codes(g)
            assert codes[0] == want[0] and sum(codes[1:]) == 0, text
        finally:
            tc.tc_graph_free(g)
