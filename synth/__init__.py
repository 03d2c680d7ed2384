"""Seeded synthetic digraphs (ctypes wrapper over ``synth.cpp``).

The workloads stand in for the thesis's real social-network datasets
(Sec. 4.1), which are not available: sparse, power-law, mean degree ~4-16.
This module draws arcs only; it holds no part of the census arithmetic, and
both the CUDA library's tests/benchmark and the CPU oracle consume its output.

Named workloads (sizes and seeds fixed here):

=====  ======================================================================
c1     directed G(n,p), n=1024, p=8/1023, each arc reciprocated w.p. 0.25
c2     R-MAT scale 20, edge factor 8, (a,b,c)=(.57,.19,.19), loops/dups
       removed, 10% of arcs reciprocated, ids permuted
c3     R-MAT scale 22, edge factor 4, every arc from higher to lower
       generator id (no mutual dyads), ids permuted
c4     4096 independent graphs, n log-uniform in [64, 65536], even index
       G(n,p) with mean out-degree U(4,32), odd index R-MAT edge factor 8,
       reciprocity U(0, 0.5)
c5     directed Chung-Lu, n=2^22, power-law exponent 2.1, mean total degree
       16, reciprocity 0.15, ids permuted; the largest expected total degree
       is set to 1.6e5 so that the largest realised degree, after loops and
       duplicate arcs are dropped, is ~1e5 (101,076)
=====  ======================================================================
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.cpp")
_LIB = os.path.join(_HERE, "libtcsynth.so")


def build(force: bool = False) -> str:
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
        P, i32, u64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
        lib.synth_gnp.argtypes = [i32, f64, f64, u64]
        lib.synth_gnp.restype = P
        lib.synth_rmat.argtypes = [i32, i32, f64, f64, f64, f64, i32, i32, u64]
        lib.synth_rmat.restype = P
        lib.synth_chung_lu.argtypes = [i32, f64, f64, f64, f64, u64]
        lib.synth_chung_lu.restype = P
        lib.synth_batch.argtypes = [i32, i32, i32, f64, f64, i32, f64, u64]
        lib.synth_batch.restype = P
        lib.synth_size.argtypes = [P, P, P]
        lib.synth_copy.argtypes = [P, P, P, P, P]
        lib.synth_free.argtypes = [P]
        _lib = lib
    return _lib


@dataclass
class Arcs:
    """Arc list of one graph (n vertices, ids in [0, n))."""
    n: int
    src: np.ndarray  # int32[m]
    dst: np.ndarray  # int32[m]

    @property
    def m(self) -> int:
        return int(self.src.size)


@dataclass
class Batch:
    """Concatenated arc lists of G graphs; graph g owns arcs goff[g]:goff[g+1]
    with local ids in [0, ns[g])."""
    ns: np.ndarray    # int32[G]
    goff: np.ndarray  # int64[G+1]
    src: np.ndarray
    dst: np.ndarray

    def graph(self, g: int) -> Arcs:
        a, b = int(self.goff[g]), int(self.goff[g + 1])
        return Arcs(int(self.ns[g]), self.src[a:b], self.dst[a:b])

    def __len__(self) -> int:
        return int(self.ns.size)


def _take(h):
    lib = _get()
    m = ctypes.c_int64()
    G = ctypes.c_int32()
    lib.synth_size(h, ctypes.byref(m), ctypes.byref(G))
    src = np.empty(m.value, dtype=np.int32)
    dst = np.empty(m.value, dtype=np.int32)
    goff = np.empty(G.value + 1, dtype=np.int64)
    gn = np.empty(G.value, dtype=np.int32)
    lib.synth_copy(h, src.ctypes.data_as(ctypes.c_void_p), dst.ctypes.data_as(ctypes.c_void_p),
                   goff.ctypes.data_as(ctypes.c_void_p), gn.ctypes.data_as(ctypes.c_void_p))
    lib.synth_free(h)
    return src, dst, goff, gn


def gnp(n: int, p: float, recip: float = 0.0, seed: int = 1) -> Arcs:
    src, dst, _, _ = _take(_get().synth_gnp(int(n), float(p), float(recip), int(seed)))
    return Arcs(int(n), src, dst)


def rmat(scale: int, edge_factor: int, a=0.57, b=0.19, c=0.19, recip=0.0,
         orient_down=False, permute=True, seed: int = 1) -> Arcs:
    src, dst, _, gn = _take(_get().synth_rmat(int(scale), int(edge_factor), a, b, c, recip,
                                              int(orient_down), int(permute), int(seed)))
    return Arcs(int(gn[0]), src, dst)


def chung_lu(n: int, gamma=2.1, mean_total_degree=16.0, max_degree=1e5, recip=0.15,
             seed: int = 1) -> Arcs:
    src, dst, _, _ = _take(_get().synth_chung_lu(int(n), gamma, mean_total_degree,
                                                 max_degree, recip, int(seed)))
    return Arcs(int(n), src, dst)


def batch(G: int, n_lo=64, n_hi=65536, deg_lo=4.0, deg_hi=32.0, edge_factor=8,
          recip_hi=0.5, seed: int = 1) -> Batch:
    src, dst, goff, gn = _take(_get().synth_batch(int(G), int(n_lo), int(n_hi), deg_lo, deg_hi,
                                                  int(edge_factor), recip_hi, int(seed)))
    return Batch(gn, goff, src, dst)


# ------------------------------------------------------------ named workloads

def c1() -> Arcs:
    return gnp(1024, 8.0 / 1023.0, recip=0.25, seed=1)


def c2() -> Arcs:
    return rmat(20, 8, recip=0.10, permute=True, seed=2)


def c3() -> Arcs:
    return rmat(22, 4, recip=0.0, orient_down=True, permute=True, seed=3)


def c4(G: int = 4096) -> Batch:
    return batch(G, 64, 65536, 4.0, 32.0, 8, 0.5, seed=4)


def c5() -> Arcs:
    return chung_lu(1 << 22, 2.1, 16.0, 1.6e5, 0.15, seed=5)


def c3s() -> Arcs:
    """Half-size c3 (R-MAT scale 21): a profiling case whose adjacency and
    task arrays still exceed the 126 MB L2."""
    return rmat(21, 4, recip=0.0, orient_down=True, permute=True, seed=3)


WORKLOADS = {"c1": c1, "c2": c2, "c3": c3, "c3s": c3s, "c4": c4, "c5": c5}
