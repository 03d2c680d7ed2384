"""Plants plausible mistakes in a copy of the oracle (on the CPU) and checks
that the pins catch every one: a transposed operand, an off-by-one in the
dyadic term, a flipped canonical test, non-canonical dyads, swapped D/U
naming, a wrong dyad type and a wrong bit weight of the pre-computed code."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "oracle.cpp")

MUTANTS = [
    ("code += 8 * (is_edge(g, w, u)", "code += 8 * (is_edge(g, u, w)"),
    ("(n - (int64_t)S.size() - 2)", "(n - (int64_t)S.size() - 1)"),
    ("u < w && !is_neighbour(g, u, w)", "u < w && is_neighbour(g, u, w)"),
    ("if (!(u < v)) continue;", "if (!(u != v)) continue;"),
    ("return asym_out[r] == 1 ? 6 : 7;", "return asym_out[r] == 1 ? 7 : 6;"),
    ("(e0 && e1) ? 2 /* 102 */ : 1", "(e0 || e1) ? 2 /* 102 */ : 1"),
    ("const int pre = e0 + 2 * e1;", "const int pre = 2 * e0 + e1;"),
    ("if (asym_out[r] == 2) return 11;", "if (asym_in[r] == 2) return 11;"),
]


def _load(path):
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.oracle_graph_new.argtypes = [ctypes.c_int32, ctypes.c_int64, P, P]
    lib.oracle_graph_new.restype = P
    lib.oracle_graph_free.argtypes = [P]
    lib.oracle_census.argtypes = [P, ctypes.c_int32, P, P]
    lib.oracle_brute.argtypes = [ctypes.c_int32, ctypes.c_int64, P, P, P]
    return lib


def _census(lib, n, src, dst):
    s = np.ascontiguousarray(src, dtype=np.int32)
    d = np.ascontiguousarray(dst, dtype=np.int32)
    h = lib.oracle_graph_new(n, s.size, s.ctypes.data_as(ctypes.c_void_p),
                             d.ctypes.data_as(ctypes.c_void_p))
    lo = np.zeros(16, np.uint64)
    hi = np.zeros(16, np.uint64)
    lib.oracle_census(h, 1, lo.ctypes.data_as(ctypes.c_void_p), hi.ctypes.data_as(ctypes.c_void_p))
    lib.oracle_graph_free(h)
    return [int(a) | (int(b) << 64) for a, b in zip(lo, hi)]


def _pins_pass(lib):
    """A reduced set of the pins: external routine on random graphs and the
    exhaustive 64 triads."""
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(5)
    for _ in range(6):
        n = int(rng.integers(6, 30))
        s, d = np.nonzero(rng.random((n, n)) < 0.2)
        keep = s != d
        s, d = s[keep], d[keep]
        G = nx.DiGraph()
        G.add_nodes_from(range(n))
        G.add_edges_from(zip(s.tolist(), d.tolist()))
        tc = nx.triadic_census(G)
        if _census(lib, n, s, d) != [tc[k] for k in oracle.TYPE_NAMES]:
            return False
    return True


def test_unmutated_copy_passes(tmp_path):
    so = tmp_path / "lib.so"
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-pthread", SRC,
                           "-o", str(so)])
    assert _pins_pass(_load(str(so)))


@pytest.mark.parametrize("k", range(len(MUTANTS)))
def test_mutant_is_caught(tmp_path, k):
    if shutil.which("g++") is None:
        pytest.skip("no compiler")
    old, new = MUTANTS[k]
    text = open(SRC).read()
    assert text.count(old) == 1, old
    cpp = tmp_path / "mut.cpp"
    cpp.write_text(text.replace(old, new))
    so = tmp_path / "mut.so"
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-pthread", str(cpp),
                           "-o", str(so)])
    assert not _pins_pass(_load(str(so))), f"mutant {k} survived: {new}"
