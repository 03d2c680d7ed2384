"""Python binding for libtc, the exact triad-census library for one B300.

This module only marshals arguments for the C-ABI in ``include/tc.h``; every
step of the census runs in the library's CUDA kernels.  Entry points keep the
C names:

    tc_graph_build, tc_graph_build_batched, tc_graph_stats, tc_graph_export,
    tc_census, tc_census_batched, tc_census_codes, tc_census_codes_batched,
    tc_graph_free, tc_opts_default,
    tc_triad_type, tc_status_str, tc_last_error

Host inputs are numpy arrays (or anything ``np.asarray`` accepts); device
inputs are CUDA torch tensors (their ``data_ptr`` is passed with the
TC_DEVICE_PTRS flag).  Census results come back as lists of 16 Python ints in
MAN order (003 012 102 021D 021U 021C 111D 111U 030T 030C 201 120D 120U 120C
210 300), the 003 count rebuilt from its two 64-bit halves; the 64-code
census (tc_census_codes) as lists of 64 ints indexed by the labelled code.

There is no CPU fallback: if ``libtc.so`` is missing, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtc.so")

TYPE_NAMES = ("003", "012", "102", "021D", "021U", "021C", "111D", "111U",
              "030T", "030C", "201", "120D", "120U", "120C", "210", "300")

TC_OK, TC_ERR_ARG, TC_ERR_ID_RANGE, TC_ERR_OOM, TC_ERR_CUDA, TC_ERR_TIMEOUT, TC_ERR_UNSUPPORTED = range(7)
TC_BIN_HEURISTIC, TC_BIN_MLP, TC_BIN_EXACT = 0, 1, 2
TC_TRI_FORWARD, TC_TRI_MERGE, TC_TRI_AUTO = 0, 1, 2
TC_DEVICE_PTRS = 1
TC_UNDIRECTED = 4
TC_OUT_DEVICE = 2

EXPORTS = ("tc_opts_default", "tc_graph_build", "tc_graph_build_batched", "tc_graph_stats",
           "tc_graph_export", "tc_census", "tc_census_batched", "tc_triad_type",
           "tc_graph_free", "tc_status_str", "tc_last_error", "tc_census_profile",
           "tc_census_csr_noalloc", "tc_plan_create", "tc_plan_run", "tc_plan_free", "tc_autotune",
           "tc_cost_sample", "tc_cost_features", "tc_mlp_loss_grad", "tc_mlp_train", "tc_mlp_predict",
           "tc_cost_model_load", "tc_census_codes", "tc_census_codes_batched",
           "tc_graph_build_text", "tc_union_sizes", "tc_path_features", "tc_path_model_load",
           "tc_path_route", "tc_census_shard", "tc_census_fold")
TC_MLP_NPARAM = 1476
TC_ACC_WORDS = 67
TC_NOALLOC_MAX_N = 262144
TC_NOALLOC_MAX_DYADS = 262144


class TcCensus(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint64 * 16), ("count003_hi", ctypes.c_uint64)]

    def to_list(self) -> list[int]:
        c = [int(x) for x in self.count]
        c[0] |= int(self.count003_hi) << 64
        return c


class TcCensus64(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint64 * 64), ("count0_hi", ctypes.c_uint64)]

    def to_list(self) -> list[int]:
        c = [int(x) for x in self.count]
        c[0] |= int(self.count0_hi) << 64
        return c


class TcStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in
                ("n", "arcs", "dyads", "mutual", "asym", "merged_entries", "max_degree")]

    def to_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class TcOpts(ctypes.Structure):
    _fields_ = [("bin_mode", ctypes.c_int32), ("thr_thread", ctypes.c_int32),
                ("thr_warp", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("split_cta", ctypes.c_int32),
                ("stream_max", ctypes.c_int32), ("persistent", ctypes.c_int32),
                ("hub_ratio", ctypes.c_int32), ("own_min", ctypes.c_int32),
                ("row_tasks", ctypes.c_int32), ("tri_path", ctypes.c_int32), ("fwd_big", ctypes.c_int32)]


class TcProfile(ctypes.Structure):
    _fields_ = [("ms_tasks", ctypes.c_float), ("ms_split", ctypes.c_float),
                ("ms_tiles", ctypes.c_float), ("ms_stream", ctypes.c_float), ("ms_owner", ctypes.c_float),
                ("ms_warp", ctypes.c_float),
                ("ms_thread", ctypes.c_float), ("ms_merge", ctypes.c_float),
                ("ms_fold", ctypes.c_float),
                ("ms_total", ctypes.c_float), ("launches", ctypes.c_int32),
                ("bin_tasks", ctypes.c_int64 * 4), ("bin_entries", ctypes.c_int64 * 4),
                ("chunks", ctypes.c_int64), ("hub_tasks", ctypes.c_int64),
                ("hub_entries", ctypes.c_int64), ("owner_items", ctypes.c_int64),
                ("owner_tasks", ctypes.c_int64), ("owner_entries", ctypes.c_int64),
                ("owner_probes", ctypes.c_int64), ("owner_staged", ctypes.c_int64),
                ("ms_forward", ctypes.c_float), ("ms_tri_map", ctypes.c_float),
                ("ms_tri_search", ctypes.c_float), ("ms_owner_prep", ctypes.c_float),
                ("fwd_entries", ctypes.c_int64), ("map_items", ctypes.c_int64),
                ("map_lookups", ctypes.c_int64), ("map_triangles", ctypes.c_int64),
                ("search_lookups", ctypes.c_int64), ("search_triangles", ctypes.c_int64),
                ("map_dyads", ctypes.c_int64), ("search_dyads", ctypes.c_int64),
                ("map_list_entries", ctypes.c_int64), ("ms_exact_cost", ctypes.c_float)]

    def to_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        for k in ("bin_tasks", "bin_entries"):
            d[k] = [int(x) for x in d[k]]
        return d


class TcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} [status {status}]")
        self.status = status


_lib = None


def load():
    """Load libtc.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libtc.so is missing ({LIB_PATH}); build it with "
                           "`python -m paper_1603_02655_b300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    P, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    lib.tc_opts_default.argtypes = [P]
    lib.tc_graph_build.argtypes = [i32, P, P, i64, u32, P, P]
    lib.tc_graph_build_batched.argtypes = [i32, P, P, P, P, u32, P, P]
    lib.tc_graph_stats.argtypes = [P, P]
    lib.tc_graph_export.argtypes = [P, P, P]
    lib.tc_census.argtypes = [P, P, P, u32, P]
    lib.tc_census_batched.argtypes = [i32, P, P, P, u32, P]
    lib.tc_census_codes.argtypes = [P, P, P, u32, P]
    lib.tc_graph_build_text.argtypes = [P, i64, i32, u32, P, P]
    lib.tc_union_sizes.argtypes = [P, P, i32, P, P]
    lib.tc_union_sizes.restype = ctypes.c_int
    lib.tc_graph_build_text.restype = ctypes.c_int
    lib.tc_census_codes_batched.argtypes = [i32, P, P, P, u32, P]
    lib.tc_triad_type.argtypes = [ctypes.c_int]
    lib.tc_triad_type.restype = ctypes.c_int
    lib.tc_census_profile.argtypes = [P]
    lib.tc_census_profile.restype = ctypes.c_int
    lib.tc_census_csr_noalloc.argtypes = [i32, P, P, i64, P, P]
    lib.tc_census_csr_noalloc.restype = ctypes.c_int
    lib.tc_plan_create.argtypes = [i32, P, P, P, P, P]
    lib.tc_plan_create.restype = ctypes.c_int
    lib.tc_plan_run.argtypes = [P, P]
    lib.tc_plan_run.restype = ctypes.c_int
    lib.tc_plan_free.argtypes = [P]
    lib.tc_plan_free.restype = None
    lib.tc_autotune.argtypes = [i32, P, P, i32, P, P, P, P]
    lib.tc_autotune.restype = ctypes.c_int
    lib.tc_cost_sample.argtypes = [i32, P, i32, i32, i32, P, P, P]
    lib.tc_cost_features.argtypes = [P, P, i32, P, P]
    lib.tc_mlp_loss_grad.argtypes = [P, P, P, P, i32, P, P, P]
    lib.tc_mlp_train.argtypes = [P, P, P, P, i32, i32, i32, ctypes.c_float, ctypes.c_uint64, P, P]
    lib.tc_mlp_predict.argtypes = [P, P, i32, i32, P, P]
    lib.tc_cost_model_load.argtypes = [P]
    lib.tc_path_features.argtypes = [i32, P, P]
    lib.tc_path_model_load.argtypes = [P]
    lib.tc_path_route.argtypes = [i32, P, P, P]
    lib.tc_census_shard.argtypes = [i32, P, P, i32, i32, P, P]
    lib.tc_census_fold.argtypes = [i32, P, P, P, P, u32, P]
    for name in ("tc_census_shard", "tc_census_fold"):
        getattr(lib, name).restype = ctypes.c_int
    for name in ("tc_path_features", "tc_path_model_load", "tc_path_route"):
        getattr(lib, name).restype = ctypes.c_int
    for name in ("tc_cost_sample", "tc_cost_features", "tc_mlp_loss_grad", "tc_mlp_train", "tc_mlp_predict",
                 "tc_cost_model_load"):
        getattr(lib, name).restype = ctypes.c_int
    lib.tc_graph_free.argtypes = [P]
    lib.tc_graph_free.restype = None
    lib.tc_status_str.argtypes = [ctypes.c_int]
    lib.tc_status_str.restype = ctypes.c_char_p
    lib.tc_last_error.argtypes = []
    lib.tc_last_error.restype = ctypes.c_char_p
    for name in ("tc_opts_default", "tc_graph_build", "tc_graph_build_batched", "tc_graph_stats",
                 "tc_graph_export", "tc_census", "tc_census_batched", "tc_census_codes",
                 "tc_census_codes_batched"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status: int, what: str):
    if status != TC_OK:
        lib = load()
        raise TcError(status, f"{what}: {lib.tc_status_str(status).decode()}: "
                              f"{lib.tc_last_error().decode()}")


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _arr(x, dtype):
    """(pointer, keepalive, is_device) for a host array or a CUDA torch tensor."""
    if hasattr(x, "is_cuda") and x.is_cuda:
        import torch
        want = {np.int32: torch.int32, np.int64: torch.int64}[dtype]
        if x.dtype != want or not x.is_contiguous():
            raise TypeError(f"device array must be a contiguous {want} tensor")
        return x.data_ptr(), x, True
    a = np.ascontiguousarray(np.asarray(x, dtype=dtype).reshape(-1))
    return a.ctypes.data, a, False


# ------------------------------------------------------------------ calls

def tc_status_str(status: int) -> str:
    return load().tc_status_str(int(status)).decode()


def tc_last_error() -> str:
    return load().tc_last_error().decode()


def tc_triad_type(code: int) -> int:
    return int(load().tc_triad_type(int(code)))


def tc_opts_default(**over) -> TcOpts:
    o = TcOpts()
    _check(load().tc_opts_default(ctypes.byref(o)), "tc_opts_default")
    for k, v in over.items():
        setattr(o, k, int(v))
    return o


def tc_graph_build(n: int, src, dst, stream=None, undirected: bool = False) -> int:
    """Build one graph; returns the opaque handle (an int).  With
    `undirected`, each pair is an edge (both arcs)."""
    ps, ks, ds = _arr(src, np.int32)
    pd, kd, dd = _arr(dst, np.int32)
    if ds != dd:
        raise TypeError("src and dst must both be host or both be device arrays")
    m = int(ks.numel() if ds else ks.size)
    if m != int(kd.numel() if dd else kd.size):
        raise ValueError("src and dst differ in length")
    h = ctypes.c_void_p()
    flags = (TC_DEVICE_PTRS if ds else 0) | (TC_UNDIRECTED if undirected else 0)
    st = load().tc_graph_build(int(n), ps if m else None, pd if m else None, m, flags, _stream(stream),
                               ctypes.byref(h))
    _check(st, "tc_graph_build")
    return h.value


def tc_graph_build_text(text, id_base: int = 1, stream=None) -> int:
    """Build one graph from a Pajek-style network file's contents (bytes or
    str on the host, or a CUDA uint8 tensor), parsed on the device."""
    if isinstance(text, str):
        text = text.encode()
    h = ctypes.c_void_p()
    if isinstance(text, (bytes, bytearray)):
        buf = ctypes.create_string_buffer(bytes(text), len(text))
        st = load().tc_graph_build_text(ctypes.cast(buf, ctypes.c_void_p), len(text), int(id_base), 0,
                                        _stream(stream), ctypes.byref(h))
    else:  # a CUDA tensor of bytes
        st = load().tc_graph_build_text(text.data_ptr(), int(text.numel()), int(id_base), TC_DEVICE_PTRS,
                                        _stream(stream), ctypes.byref(h))
    _check(st, "tc_graph_build_text")
    return h.value


def tc_graph_build_batched(ns, arc_off, src, dst, stream=None, undirected: bool = False) -> list[int]:
    """Build G graphs (ids local to each graph); returns G handles."""
    ns = np.ascontiguousarray(np.asarray(ns, dtype=np.int32))
    off = np.ascontiguousarray(np.asarray(arc_off, dtype=np.int64))
    G = int(ns.size)
    if off.size != G + 1:
        raise ValueError("arc_off must have G+1 entries")
    ps, ks, ds = _arr(src, np.int32)
    pd, kd, dd = _arr(dst, np.int32)
    if ds != dd:
        raise TypeError("src and dst must both be host or both be device arrays")
    out = (ctypes.c_void_p * G)()
    flags = (TC_DEVICE_PTRS if ds else 0) | (TC_UNDIRECTED if undirected else 0)
    st = load().tc_graph_build_batched(G, ns.ctypes.data, off.ctypes.data, ps, pd, flags, _stream(stream), out)
    _check(st, "tc_graph_build_batched")
    return [out[i] for i in range(G)]


def tc_graph_stats(g: int) -> dict:
    s = TcStats()
    _check(load().tc_graph_stats(g, ctypes.byref(s)), "tc_graph_stats")
    return s.to_dict()


def tc_graph_export(g: int):
    """(row_ptr int64[n+1], adj uint32[2*dyads]) copied to host."""
    st = tc_graph_stats(g)
    rp = np.zeros(st["n"] + 1, dtype=np.int64)
    adj = np.zeros(max(1, 2 * st["dyads"]), dtype=np.uint32)
    _check(load().tc_graph_export(g, rp.ctypes.data, adj.ctypes.data), "tc_graph_export")
    return rp, adj[: 2 * st["dyads"]]


def tc_census(g: int, opts: TcOpts | None = None, out=None, stream=None):
    """Census of one graph.  Without `out`: host result, a list of 16 ints.
    With `out` (a CUDA tensor of >= 17 int64): asynchronous device result."""
    lib = load()
    po = ctypes.byref(opts) if opts is not None else None
    if out is None:
        c = TcCensus()
        _check(lib.tc_census(g, po, ctypes.byref(c), 0, _stream(stream)), "tc_census")
        return c.to_list()
    _check(lib.tc_census(g, po, out.data_ptr(), TC_OUT_DEVICE, _stream(stream)), "tc_census")
    return out


def tc_census_batched(gs, opts: TcOpts | None = None, out=None, stream=None):
    """Censuses of graphs `gs` (handles of one batched build).  Without `out`:
    list of per-graph lists; with `out` (CUDA tensor of >= 17*G int64):
    asynchronous device result."""
    lib = load()
    G = len(gs)
    arr = (ctypes.c_void_p * max(G, 1))(*gs)
    po = ctypes.byref(opts) if opts is not None else None
    if out is None:
        res = (TcCensus * max(G, 1))()
        _check(lib.tc_census_batched(G, arr, po, res, 0, _stream(stream)), "tc_census_batched")
        return [res[i].to_list() for i in range(G)]
    _check(lib.tc_census_batched(G, arr, po, out.data_ptr(), TC_OUT_DEVICE, _stream(stream)),
           "tc_census_batched")
    return out


def _device_words(t, need, what):
    """A CUDA int64 tensor of at least `need` elements, contiguous (checked
    here: the library reads and writes `need` words through its pointer)."""
    if not (hasattr(t, "is_cuda") and t.is_cuda) or str(t.dtype) != "torch.int64" or not t.is_contiguous() \
            or t.numel() < need:
        raise TcError(TC_ERR_ARG, f"{what}: need a contiguous CUDA int64 tensor of >= {need} elements")
    return t.data_ptr()


def tc_census_shard(gs, shard: int, nshards: int, acc, opts: TcOpts | None = None, stream=None):
    """Shard `shard` of `nshards` of the census of graphs `gs` (one build):
    the raw accumulators of graph i go to acc[i*TC_ACC_WORDS:(i+1)*TC_ACC_WORDS]
    (CUDA int64 tensor, asynchronous).  Summed over all shards (int64 sums wrap
    like the library's uint64 words) and folded with tc_census_fold, they give
    tc_census_batched's result."""
    lib = load()
    G = len(gs)
    arr = (ctypes.c_void_p * max(G, 1))(*gs)
    po = ctypes.byref(opts) if opts is not None else None
    ptr = _device_words(acc, TC_ACC_WORDS * G, "tc_census_shard") if G else None
    _check(lib.tc_census_shard(G, arr, po, int(shard), int(nshards), ptr, _stream(stream)), "tc_census_shard")
    return acc


def tc_census_fold(gs, acc, out=None, stream=None):
    """Fold summed shard accumulators (CUDA int64 tensor, TC_ACC_WORDS per
    graph) into censuses: host lists without `out`, else into `out` (CUDA
    tensor of >= 17*G int64, asynchronous)."""
    lib = load()
    G = len(gs)
    arr = (ctypes.c_void_p * max(G, 1))(*gs)
    ptr = _device_words(acc, TC_ACC_WORDS * G, "tc_census_fold") if G else None
    if out is None:
        res = (TcCensus * max(G, 1))()
        _check(lib.tc_census_fold(G, arr, ptr, res, None, 0, _stream(stream)), "tc_census_fold")
        return [res[i].to_list() for i in range(G)]
    _check(lib.tc_census_fold(G, arr, ptr, _device_words(out, 17 * G, "tc_census_fold"), None, TC_OUT_DEVICE,
                              _stream(stream)), "tc_census_fold")
    return out


def tc_census_codes(g: int, opts: TcOpts | None = None, out=None, stream=None):
    """64-code census of one graph.  Without `out`: host result, a list of 64
    ints (index = labelled code).  With `out` (a CUDA tensor of >= 65 int64):
    asynchronous device result."""
    lib = load()
    po = ctypes.byref(opts) if opts is not None else None
    if out is None:
        c = TcCensus64()
        _check(lib.tc_census_codes(g, po, ctypes.byref(c), 0, _stream(stream)), "tc_census_codes")
        return c.to_list()
    _check(lib.tc_census_codes(g, po, out.data_ptr(), TC_OUT_DEVICE, _stream(stream)), "tc_census_codes")
    return out


def tc_census_codes_batched(gs, opts: TcOpts | None = None, stream=None):
    """64-code censuses of graphs `gs` (handles of one batched build), host
    result: one list of 64 ints per graph."""
    lib = load()
    G = len(gs)
    arr = (ctypes.c_void_p * max(G, 1))(*gs)
    po = ctypes.byref(opts) if opts is not None else None
    res = (TcCensus64 * max(G, 1))()
    _check(lib.tc_census_codes_batched(G, arr, po, res, 0, _stream(stream)), "tc_census_codes_batched")
    return [res[i].to_list() for i in range(G)]


def tc_census_profile() -> dict:
    """Kernel times and bin counts of this thread's last profiled census."""
    p = TcProfile()
    _check(load().tc_census_profile(ctypes.byref(p)), "tc_census_profile")
    return p.to_dict()


def tc_census_csr_noalloc(n: int, row_ptr, adj, nnz: int, out, stream=None):
    """Census of a caller-held device CSR (row_ptr int64[n+1], adj 32-bit
    [nnz] CUDA tensors) into `out` (CUDA int64 tensor of >= 17 words), using
    only the library's fixed scratch area: no device allocation.  The
    tensors are checked here (device, dtype, contiguity, length) so that the
    kernels never read or write past them."""
    def need(ok, what):
        if not ok:
            raise TcError(TC_ERR_ARG, "tc_census_csr_noalloc: " + what)
    import torch
    need(int(n) >= 0 and int(nnz) >= 0, "negative size")
    for name, t, dts in (("row_ptr", row_ptr, (torch.int64,)), ("adj", adj, (torch.int32, torch.uint32)),
                         ("out", out, (torch.int64, torch.uint64))):
        need(isinstance(t, torch.Tensor) and t.is_cuda, f"{name} must be a CUDA tensor")
        need(t.dtype in dts, f"{name} has dtype {t.dtype}")
        need(t.is_contiguous(), f"{name} must be contiguous")
    need(row_ptr.numel() >= int(n) + 1, "row_ptr holds fewer than n+1 offsets")
    need(adj.numel() >= int(nnz), "adj holds fewer than nnz entries")
    need(out.numel() >= 17, "out holds fewer than 17 words")
    p_adj = adj.data_ptr() if nnz else None
    st = load().tc_census_csr_noalloc(int(n), row_ptr.data_ptr(), p_adj, int(nnz), out.data_ptr(),
                                      _stream(stream))
    _check(st, "tc_census_csr_noalloc")
    return out


def tc_plan_create(gs, out, opts: TcOpts | None = None, stream=None) -> int:
    """Record the census of graphs `gs` (one batched build) as a CUDA graph
    writing to `out` (CUDA int64 tensor of >= 17*len(gs) words)."""
    G = len(gs)
    arr = (ctypes.c_void_p * max(G, 1))(*gs)
    h = ctypes.c_void_p()
    po = ctypes.byref(opts) if opts is not None else None
    _check(load().tc_plan_create(G, arr, po, out.data_ptr(), _stream(stream), ctypes.byref(h)),
           "tc_plan_create")
    return h.value


def tc_plan_run(plan: int, stream=None) -> None:
    _check(load().tc_plan_run(plan, _stream(stream)), "tc_plan_run")


def tc_plan_free(plan: int) -> None:
    if plan:
        load().tc_plan_free(plan)


def tc_autotune(gs, base: TcOpts | None = None, max_trials: int = 0, stream=None):
    """(best options, their census time in ms, options timed) for graphs gs."""
    G = len(gs)
    arr = (ctypes.c_void_p * max(G, 1))(*gs)
    best = TcOpts()
    ms = ctypes.c_float()
    n = ctypes.c_int32()
    pb = ctypes.byref(base) if base is not None else None
    _check(load().tc_autotune(G, arr, pb, int(max_trials), _stream(stream), ctypes.byref(best),
                              ctypes.byref(ms), ctypes.byref(n)), "tc_autotune")
    return best, float(ms.value), int(n.value)


TUNED_FIELDS = ("bin_mode", "thr_thread", "thr_warp", "chunk", "split_cta", "stream_max", "persistent",
                "hub_ratio", "own_min", "tri_path", "fwd_big")


def graph_class(stats: list) -> str:
    """Coarse class of a list of graphs for the autotune cache: count,
    total merged entries, mean task length and largest degree (log2 buckets)."""
    import math
    G = len(stats)
    merged = sum(s["merged_entries"] for s in stats)
    dyads = sum(s["dyads"] for s in stats)
    maxd = max((s["max_degree"] for s in stats), default=0)
    lg = lambda x: int(round(math.log2(x))) if x > 0 else 0  # noqa: E731
    return f"G{lg(G)}-m{lg(merged)}-t{lg(merged / dyads) if dyads else 0}-d{lg(maxd)}"


def autotune(gs, cache_path: str | None = None, base: TcOpts | None = None, max_trials: int = 0,
             stream=None, retune: bool = False) -> TcOpts:
    """Autotuned census options for graphs gs, cached as JSON per device name
    and graph class (default file: $TC_AUTOTUNE_CACHE or
    ~/.cache/tc_b300/autotune.json)."""
    import json
    import torch
    path = cache_path or os.environ.get("TC_AUTOTUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "tc_b300", "autotune.json")
    dev = torch.cuda.get_device_name()
    key = graph_class([tc_graph_stats(g) for g in gs])
    cache = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    hit = cache.get(dev, {}).get(key)
    if hit and not retune and all(k in hit for k in TUNED_FIELDS):
        return tc_opts_default(**{k: hit[k] for k in TUNED_FIELDS})
    best, ms, trials = tc_autotune(gs, base, max_trials, stream)
    entry = {k: int(getattr(best, k)) for k in TUNED_FIELDS}
    entry.update(ms=ms, trials=trials)
    cache.setdefault(dev, {})[key] = entry
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return best


def tc_cost_sample(gs, bin_: int, mask: int, cap: int, stream=None):
    """Instrumented census with every eligible task forced into bin `bin_`:
    an int32 CUDA tensor [n, 4] of {u, v, bin, cycles} records."""
    import torch
    G = len(gs)
    arr = (ctypes.c_void_p * max(G, 1))(*gs)
    buf = torch.zeros((max(cap, 1), 4), dtype=torch.int32, device="cuda")
    n = ctypes.c_int32()
    _check(load().tc_cost_sample(G, arr, int(bin_), int(mask), int(cap), buf.data_ptr(), ctypes.byref(n),
                                 _stream(stream)), "tc_cost_sample")
    return buf[: n.value]


def tc_cost_features(g: int, uv, stream=None):
    """Features float32 CUDA tensor [n, 8] of tasks uv (int32 CUDA tensor [n, 2])."""
    import torch
    uv = uv.contiguous()
    out = torch.empty((uv.shape[0], 8), dtype=torch.float32, device="cuda")
    _check(load().tc_cost_features(g, uv.data_ptr(), int(uv.shape[0]), out.data_ptr(), _stream(stream)),
           "tc_cost_features")
    return out


def tc_union_sizes(g: int, uv, stream=None):
    """|S| = |N(u) u N(v) minus {u, v}| (int32 CUDA tensor [n]) of pairs uv
    (int32 CUDA tensor [n, 2], global rows of one graph of g's build each)."""
    import torch
    uv = uv.contiguous()
    out = torch.empty(uv.shape[0], dtype=torch.int32, device="cuda")
    _check(load().tc_union_sizes(g, uv.data_ptr(), int(uv.shape[0]), out.data_ptr(), _stream(stream)),
           "tc_union_sizes")
    return out


def tc_mlp_loss_grad(params, feat, bins, target, stream=None):
    """(loss, gradient) of the cost-model loss; CUDA tensors in, FP32 out."""
    import torch
    grad = torch.empty(TC_MLP_NPARAM, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    _check(load().tc_mlp_loss_grad(params.data_ptr(), feat.data_ptr(), bins.data_ptr(), target.data_ptr(),
                                   int(feat.shape[0]), grad.data_ptr(), loss.data_ptr(), _stream(stream)),
           "tc_mlp_loss_grad")
    return float(loss.item()), grad


def tc_mlp_train(params, feat, bins, target, steps: int, batch: int, lr: float, seed: int = 1, stream=None):
    """Adam steps on `params` (float32 CUDA tensor, updated in place); returns
    the loss over all samples at the end."""
    import torch
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    _check(load().tc_mlp_train(params.data_ptr(), feat.data_ptr(), bins.data_ptr(), target.data_ptr(),
                               int(feat.shape[0]), int(steps), int(batch), float(lr), int(seed),
                               loss.data_ptr(), _stream(stream)), "tc_mlp_train")
    return float(loss.item())


def tc_mlp_predict(params, feat, half_precision: bool = True, stream=None):
    import torch
    out = torch.empty((feat.shape[0], 4), dtype=torch.float32, device="cuda")
    _check(load().tc_mlp_predict(params.data_ptr(), feat.data_ptr(), int(feat.shape[0]), int(half_precision),
                                 out.data_ptr(), _stream(stream)), "tc_mlp_predict")
    return out


def tc_cost_model_load(params) -> None:
    """Install cost-model parameters (host float32, 1476 values) on the
    current device for TC_BIN_MLP; None uninstalls."""
    if params is None:
        _check(load().tc_cost_model_load(None), "tc_cost_model_load")
        return
    a = np.ascontiguousarray(np.asarray(params, dtype=np.float32).reshape(-1))
    if a.size != TC_MLP_NPARAM:
        raise ValueError(f"expected {TC_MLP_NPARAM} parameters")
    _check(load().tc_cost_model_load(a.ctypes.data), "tc_cost_model_load")


def _handles(gs):
    arr = (ctypes.c_void_p * max(1, len(gs)))()
    for i, g in enumerate(gs):
        arr[i] = g
    return arr


def tc_path_features(gs) -> np.ndarray:
    """Routing features float32[G, 8] of graphs of one build (host)."""
    out = np.zeros((len(gs), 8), dtype=np.float32)
    _check(load().tc_path_features(len(gs), _handles(gs), out.ctypes.data), "tc_path_features")
    return out


def tc_path_model_load(params) -> None:
    """Install the path-routing model (host float32, 1476 values: output 0 =
    log2 time on the forward path, 1 = on the merge path) on the current
    device for TC_TRI_AUTO; None uninstalls (the degree-skew rule routes)."""
    if params is None:
        _check(load().tc_path_model_load(None), "tc_path_model_load")
        return
    a = np.ascontiguousarray(np.asarray(params, dtype=np.float32).reshape(-1))
    if a.size != TC_MLP_NPARAM:
        raise ValueError(f"expected {TC_MLP_NPARAM} parameters")
    _check(load().tc_path_model_load(a.ctypes.data), "tc_path_model_load")


def tc_path_route(gs, stream=None) -> list[int]:
    """The path (TC_TRI_FORWARD or TC_TRI_MERGE) each graph takes under
    TC_TRI_AUTO."""
    out = np.zeros(len(gs), dtype=np.int32)
    _check(load().tc_path_route(len(gs), _handles(gs), out.ctypes.data, _stream(stream)), "tc_path_route")
    return [int(x) for x in out]


def tc_graph_free(g: int) -> None:
    if g:
        load().tc_graph_free(g)


def census_from_device_words(words) -> list[int]:
    """Decode one 17-word device census (int64 tensor/array) into 16 ints."""
    w = [int(x) & ((1 << 64) - 1) for x in words[:17]]
    c = w[:16]
    c[0] |= w[16] << 64
    return c


class Graph:
    """Owning wrapper around a tc_graph handle."""

    def __init__(self, n: int, src, dst, stream=None):
        self.n = int(n)
        self.h = tc_graph_build(n, src, dst, stream)

    def stats(self) -> dict:
        return tc_graph_stats(self.h)

    def census(self, opts=None, out=None, stream=None):
        return tc_census(self.h, opts, out, stream)

    def close(self):
        if self.h:
            tc_graph_free(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
