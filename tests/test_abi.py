"""C-ABI checks that need no GPU: the library builds and loads, exports every
function include/tc.h declares, and its host-only calls behave."""
import ctypes
import os
import re

import pytest

import oracle
import paper_1603_02655_b300 as tc
from paper_1603_02655_b300 import build as tcbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "tc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tc_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    tcbuild.build()
    return tc.load()


def test_exports_every_declared_symbol(lib):
    names = header_functions()
    assert len(names) >= 11
    for name in names:
        assert hasattr(lib, name), name
    # the Python binding wraps exactly the declared entry points, each with
    # its argument types declared (an undeclared pointer argument would be
    # passed as a 32-bit int)
    assert set(names) == set(tc.EXPORTS)
    for name in names:
        assert getattr(lib, name).argtypes is not None, name


def test_library_table_matches_oracle_table(lib):
    assert [tc.tc_triad_type(c) for c in range(64)] == oracle.triad_table()
    assert tc.tc_triad_type(-1) == -1 and tc.tc_triad_type(64) == -1


def test_status_strings_and_defaults(lib):
    for s in range(7):
        assert tc.tc_status_str(s).startswith("TC_")
    o = tc.tc_opts_default()
    assert o.bin_mode == tc.TC_BIN_HEURISTIC
    assert 0 <= o.thr_thread <= o.thr_warp and o.chunk >= 256


def test_argument_errors_need_no_device(lib):
    h = ctypes.c_void_p()
    assert lib.tc_graph_build(-1, None, None, 0, 0, None, ctypes.byref(h)) == tc.TC_ERR_ARG
    assert lib.tc_graph_build(5, None, None, -3, 0, None, ctypes.byref(h)) == tc.TC_ERR_ARG
    assert lib.tc_graph_build(5, None, None, 4, 0, None, ctypes.byref(h)) == tc.TC_ERR_ARG
    assert lib.tc_graph_build(1 << 30, None, None, 0, 0, None, ctypes.byref(h)) == tc.TC_ERR_UNSUPPORTED
    assert lib.tc_graph_build(5, None, None, 0, 0x80, None, ctypes.byref(h)) == tc.TC_ERR_ARG
    assert lib.tc_census(None, None, None, 0, None) == tc.TC_ERR_ARG
    assert lib.tc_census_batched(-1, None, None, None, 0, None) == tc.TC_ERR_ARG
    assert lib.tc_census_batched(0, None, None, None, 0, None) == tc.TC_OK
    assert lib.tc_census_codes(None, None, None, 0, None) == tc.TC_ERR_ARG
    assert lib.tc_census_codes_batched(-1, None, None, None, 0, None) == tc.TC_ERR_ARG
    assert lib.tc_census_codes_batched(0, None, None, None, 0, None) == tc.TC_OK
    assert lib.tc_graph_build_text(None, 0, 1, 0, None, None) == tc.TC_ERR_ARG
    assert lib.tc_union_sizes(None, None, 1, None, None) == tc.TC_ERR_ARG
    assert lib.tc_graph_build_text(b"*Vertices 3\n", 12, 2, 0, None, ctypes.byref(h)) == tc.TC_ERR_ARG
    assert lib.tc_graph_build_text(b"*Vertices 3\n", 12, 1, 0x80, None, ctypes.byref(h)) == tc.TC_ERR_ARG
    assert lib.tc_graph_build_text(None, 0, 1, 0, None, ctypes.byref(h)) == tc.TC_ERR_ARG  # empty file
    assert lib.tc_graph_build(5, None, None, 0, 0x80 | tc.TC_UNDIRECTED, None, ctypes.byref(h)) == tc.TC_ERR_ARG
    assert lib.tc_census_shard(-1, None, None, 0, 1, None, None) == tc.TC_ERR_ARG
    assert lib.tc_census_shard(0, None, None, 0, 0, None, None) == tc.TC_ERR_ARG
    assert lib.tc_census_shard(0, None, None, 3, 2, None, None) == tc.TC_ERR_ARG
    assert lib.tc_census_shard(0, None, None, 1, 2, None, None) == tc.TC_OK
    assert lib.tc_census_shard(1, None, None, 0, 1, None, None) == tc.TC_ERR_ARG
    assert lib.tc_census_fold(-1, None, None, None, None, 0, None) == tc.TC_ERR_ARG
    assert lib.tc_census_fold(0, None, None, None, None, 0, None) == tc.TC_OK
    assert lib.tc_census_fold(0, None, None, None, None, 0x80, None) == tc.TC_ERR_ARG
    assert lib.tc_graph_stats(None, None) == tc.TC_ERR_ARG
    assert lib.tc_opts_default(None) == tc.TC_ERR_ARG
    assert "null" in tc.tc_last_error() or tc.tc_last_error()
    lib.tc_graph_free(None)


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(tc, "_lib", None)
    monkeypatch.setattr(tc, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError):
        tc.load()


def test_noalloc_binding_refuses_host_or_short_tensors(lib):
    """The binding checks device, dtype and length before the call reaches
    the library (a short or host tensor would be read past its end)."""
    import torch
    rp = torch.zeros(4, dtype=torch.int64)
    adj = torch.zeros(2, dtype=torch.int32)
    out = torch.zeros(17, dtype=torch.int64)
    for args in ((3, rp, adj, 2, out), (3, rp.int(), adj, 2, out), (9, rp, adj, 2, out),
                 (3, rp, adj, 6, out), (3, rp, adj, 2, out[:5])):
        with pytest.raises(tc.TcError) as e:
            tc.tc_census_csr_noalloc(*args)
        assert e.value.status == tc.TC_ERR_ARG


def test_shard_binding_refuses_host_or_short_accumulators(lib):
    """The accumulator tensor is checked before the call reaches the library
    (TC_ACC_WORDS int64 words per graph, on the device)."""
    import torch
    for acc in (torch.zeros(tc.TC_ACC_WORDS, dtype=torch.int64), torch.zeros(tc.TC_ACC_WORDS, dtype=torch.int32)):
        with pytest.raises(tc.TcError) as e:
            tc.tc_census_shard([1], 0, 1, acc)
        assert e.value.status == tc.TC_ERR_ARG
        with pytest.raises(tc.TcError) as e:
            tc.tc_census_fold([1], acc)
        assert e.value.status == tc.TC_ERR_ARG
