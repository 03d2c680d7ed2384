"""Plants plausible mistakes in a copy of the oracle (on the CPU) and checks
that the pins catch every one: a transposed operand, an off-by-one in the
dyadic term, a flipped canonical test, non-canonical dyads, swapped D/U
naming, a wrong dyad type and a wrong bit weight of the pre-computed code;
and the same kinds of mistakes in the 64-code census loop."""
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


# the same lines in the 64-code loop (their second occurrence in the file)
CODE_MUTANTS = [
    ("code += 8 * (is_edge(g, w, u)", "code += 8 * (is_edge(g, u, w)"),
    ("u < w && !is_neighbour(g, u, w)", "u < w && is_neighbour(g, u, w)"),
    ("if (!(u < v)) continue;", "if (!(u != v)) continue;"),
    ("c[pre] += (u128)(uint64_t)(n - (int64_t)S.size() - 2);", "c[pre] += (u128)(uint64_t)(n - (int64_t)S.size() - 1);"),
    ("+ 2 * (is_edge(g, v, u) ? 1 : 0);", "+ 2 * (is_edge(g, u, v) ? 1 : 0);"),
]


def _replace_nth(text, old, new, nth):
    at = -1
    for _ in range(nth + 1):
        at = text.index(old, at + 1)
    return text[:at] + new + text[at + len(old):]


def _codes_pins_pass(lib):
    """The 64-code census against the O(n^3) definition on random graphs."""
    P = ctypes.c_void_p
    lib.oracle_census_codes.argtypes = [P, P, P]
    lib.oracle_brute_codes.argtypes = [ctypes.c_int32, ctypes.c_int64, P, P, P]
    rng = np.random.default_rng(8)
    for _ in range(6):
        n = int(rng.integers(6, 30))
        s, d = np.nonzero(rng.random((n, n)) < 0.25)
        s = np.ascontiguousarray(s, dtype=np.int32)
        d = np.ascontiguousarray(d, dtype=np.int32)
        want = np.zeros(64, np.uint64)
        if lib.oracle_brute_codes(n, s.size, s.ctypes.data_as(P), d.ctypes.data_as(P), want.ctypes.data_as(P)):
            return False
        h = lib.oracle_graph_new(n, s.size, s.ctypes.data_as(P), d.ctypes.data_as(P))
        lo = np.zeros(64, np.uint64)
        hi = np.zeros(64, np.uint64)
        lib.oracle_census_codes(h, lo.ctypes.data_as(P), hi.ctypes.data_as(P))
        lib.oracle_graph_free(h)
        if not (np.array_equal(lo, want) and not hi.any()):
            return False
    return True


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
    assert text.count(old) in (1, 2), old  # the first occurrence is the 16-type loop
    cpp = tmp_path / "mut.cpp"
    cpp.write_text(_replace_nth(text, old, new, 0))
    so = tmp_path / "mut.so"
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-pthread", str(cpp),
                           "-o", str(so)])
    assert not _pins_pass(_load(str(so))), f"mutant {k} survived: {new}"


def test_unmutated_copy_passes_codes(tmp_path):
    so = tmp_path / "lib.so"
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-pthread", SRC,
                           "-o", str(so)])
    assert _codes_pins_pass(_load(str(so)))


@pytest.mark.parametrize("k", range(len(CODE_MUTANTS)))
def test_code_mutant_is_caught(tmp_path, k):
    if shutil.which("g++") is None:
        pytest.skip("no compiler")
    old, new = CODE_MUTANTS[k]
    text = open(SRC).read()
    nth = text.count(old) - 1  # the 64-code loop follows the 16-type one
    assert nth in (0, 1), old
    cpp = tmp_path / "mut.cpp"
    cpp.write_text(_replace_nth(text, old, new, nth))
    so = tmp_path / "mut.so"
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-pthread", str(cpp),
                           "-o", str(so)])
    assert not _codes_pins_pass(_load(str(so))), f"code mutant {k} survived: {new}"
