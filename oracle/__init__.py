"""Triad-census ORACLE -- test infrastructure only.

A ctypes wrapper over ``oracle.cpp``: a plain CPU restatement of the
subquadratic triad census (thesis Sec. 2.2, Fig. "Subquadratic Triad Census
Algorithm", with the v0.4 pre-computed dyad code of Sec. 4.2.4) plus the O(n^3)
definition it must agree with.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package; the CUDA
library shares no code with it and never calls it.

Counts are returned as Python ints (exact, 128-bit on the C side), in MAN
order: 003 012 102 021D 021U 021C 111D 111U 030T 030C 201 120D 120U 120C 210
300.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

TYPE_NAMES = ("003", "012", "102", "021D", "021U", "021C", "111D", "111U",
              "030T", "030C", "201", "120D", "120U", "120C", "210", "300")


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to its source if it is missing or stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _get():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        lib.oracle_triad_table.argtypes = [P]
        lib.oracle_brute.argtypes = [i32, i64, P, P, P]
        lib.oracle_brute.restype = ctypes.c_int
        lib.oracle_graph_new.argtypes = [i32, i64, P, P]
        lib.oracle_graph_new.restype = P
        lib.oracle_graph_free.argtypes = [P]
        lib.oracle_graph_stats.argtypes = [P, P]
        lib.oracle_common.argtypes = [P, i32, i32]
        lib.oracle_common.restype = i64
        lib.oracle_census_range.argtypes = [P, i32, i32, P, P]
        lib.oracle_census_range.restype = u64
        lib.oracle_census.argtypes = [P, i32, P, P]
        lib.oracle_brute_codes.argtypes = [i32, i64, P, P, P]
        lib.oracle_brute_codes.restype = ctypes.c_int
        lib.oracle_census_codes.argtypes = [P, P, P]
        _lib = lib
    return _lib


def _arcs(src, dst):
    s = np.ascontiguousarray(np.asarray(src, dtype=np.int32).reshape(-1))
    d = np.ascontiguousarray(np.asarray(dst, dtype=np.int32).reshape(-1))
    if s.shape != d.shape:
        raise ValueError("src and dst differ in length")
    return s, d


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def triad_table() -> list[int]:
    """The 64 -> 16 map, derived from the MAN naming rules (Sec. 2.2)."""
    out = np.zeros(64, dtype=np.int32)
    _get().oracle_triad_table(_p(out))
    return [int(x) for x in out]


def brute_census(n: int, src, dst) -> list[int]:
    """O(n^3) census by definition (n <= 4096)."""
    s, d = _arcs(src, dst)
    out = np.zeros(16, dtype=np.uint64)
    if _get().oracle_brute(int(n), s.size, _p(s), _p(d), _p(out)) != 0:
        raise ValueError("oracle_brute: bad arguments")
    return [int(x) for x in out]


def brute_census_codes(n: int, src, dst) -> list[int]:
    """O(n^3) 64-code census by definition (n <= 4096); raises if some triple
    is not counted exactly once."""
    s, d = _arcs(src, dst)
    out = np.zeros(64, dtype=np.uint64)
    r = _get().oracle_brute_codes(int(n), s.size, _p(s), _p(d), _p(out))
    if r == -2:
        raise AssertionError("oracle_brute_codes: a triple is not counted exactly once")
    if r != 0:
        raise ValueError("oracle_brute_codes: bad arguments")
    return [int(x) for x in out]


def _join(lo, hi):
    return [int(l) | (int(h) << 64) for l, h in zip(lo, hi)]


class Graph:
    """Oracle CRS graph (sorted neighbour lists N(u) and out-arc lists E(u))."""

    def __init__(self, n: int, src, dst):
        s, d = _arcs(src, dst)
        self.n = int(n)
        self._h = _get().oracle_graph_new(self.n, s.size, _p(s), _p(d))
        if not self._h:
            raise ValueError("oracle graph: id out of range or bad size")

    def close(self):
        if getattr(self, "_h", None):
            _get().oracle_graph_free(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def stats(self) -> dict:
        st = np.zeros(7, dtype=np.int64)
        _get().oracle_graph_stats(self._h, _p(st))
        keys = ("n", "arcs", "dyads", "mutual", "asym", "merged_entries", "max_degree")
        return {k: int(v) for k, v in zip(keys, st)}

    def common(self, u: int, v: int) -> int:
        """|N(u) & N(v)|."""
        return int(_get().oracle_common(self._h, int(u), int(v)))

    def census(self, threads: int = 1) -> list[int]:
        """Full 16-type census (Fig. "Subquadratic Triad Census Algorithm")."""
        lo = np.zeros(16, dtype=np.uint64)
        hi = np.zeros(16, dtype=np.uint64)
        _get().oracle_census(self._h, int(threads), _p(lo), _p(hi))
        return _join(lo, hi)

    def census_codes(self) -> list[int]:
        """64-code census (Fig. "Triad Code Algorithm" without TriadTable)."""
        lo = np.zeros(64, dtype=np.uint64)
        hi = np.zeros(64, dtype=np.uint64)
        _get().oracle_census_codes(self._h, _p(lo), _p(hi))
        return _join(lo, hi)

    def census_range(self, u_begin: int, u_end: int):
        """Types 1..15 from canonical dyads with u in [u_begin, u_end) (no 003
        closure); returns (counts, merged entries processed)."""
        lo = np.zeros(16, dtype=np.uint64)
        hi = np.zeros(16, dtype=np.uint64)
        e = _get().oracle_census_range(self._h, int(u_begin), int(u_end), _p(lo), _p(hi))
        return _join(lo, hi), int(e)


def census(n: int, src, dst, threads: int = 1) -> list[int]:
    g = Graph(n, src, dst)
    try:
        return g.census(threads)
    finally:
        g.close()


def census_codes(n: int, src, dst) -> list[int]:
    g = Graph(n, src, dst)
    try:
        return g.census_codes()
    finally:
        g.close()


def choose3(n: int) -> int:
    return n * (n - 1) * (n - 2) // 6 if n >= 3 else 0
