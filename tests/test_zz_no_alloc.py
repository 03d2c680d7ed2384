"""The allocation-free census entry point (tc_census_csr_noalloc).

Callers that may not allocate device memory (their memory manager owns the
GPU, or allocation is forbidden after start-up) pass a CSR they already hold
and get the census computed in the library's fixed scratch area.  The
results are checked against the CPU oracle (and, for c1, the census the
oracle stored under tests/golden/), on two calls in a row, because the
scratch keeps the previous call's contents.  This file is collected last on
purpose, and also passes when run alone in a fresh process.
"""
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


@pytest.fixture(scope="module", autouse=True)
def lib(cuda_ok):
    tcbuild.build()
    return tc.load()


def graphs():
    rng = np.random.default_rng(21)
    yield "c1", synth.c1()
    # hubs: dyads of |N(u)|+|N(v)| in the thousands, plus sparse random arcs
    n = 6000
    src, dst = [], []
    for h in range(3):
        nb = rng.choice(n, size=2500, replace=False)
        out = rng.random(nb.size) < 0.5
        src.append(np.where(out, h, nb))
        dst.append(np.where(out, nb, h))
    src.append(rng.integers(0, n, 20000))
    dst.append(rng.integers(0, n, 20000))
    s = np.concatenate(src).astype(np.int32)
    d = np.concatenate(dst).astype(np.int32)
    rec = rng.random(s.size) < 0.3
    yield "hubs", synth.Arcs(n, np.concatenate([s, d[rec]]), np.concatenate([d, s[rec]]))
    yield "empty", synth.Arcs(10, np.zeros(0, np.int32), np.zeros(0, np.int32))


def device_csr(arcs):
    """The graph's CSR in the layout tc_graph_build writes, copied into
    caller-owned CUDA tensors (the graph handle is released first)."""
    import torch
    g = tc.tc_graph_build(arcs.n, arcs.src, arcs.dst)
    try:
        rp, adj = tc.tc_graph_export(g)
    finally:
        tc.tc_graph_free(g)
    return (torch.from_numpy(rp).cuda(), torch.from_numpy(adj.view(np.int32).copy()).cuda(), int(rp[-1]))


@pytest.mark.parametrize("case", ["c1", "hubs", "empty"])
def test_noalloc_matches_oracle_on_two_calls_in_a_row(case):
    import torch
    arcs = dict(graphs())[case]
    want = oracle.census(arcs.n, arcs.src, arcs.dst)
    if case == "c1":
        assert want == json.load(open(os.path.join(GOLDEN, "census_c1.json")))["census"]
    rp, adj, nnz = device_csr(arcs)
    out = torch.zeros(17, dtype=torch.int64, device="cuda")
    for _ in range(2):  # the scratch keeps the last call's contents
        tc.tc_census_csr_noalloc(arcs.n, rp, adj, nnz, out)
        assert tc.census_from_device_words(out.cpu().tolist()) == want


def test_noalloc_rejects_sizes_beyond_the_maximum():
    import torch
    rp = torch.zeros(tc.TC_NOALLOC_MAX_N + 2, dtype=torch.int64, device="cuda")
    adj = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.zeros(17, dtype=torch.int64, device="cuda")
    with pytest.raises(tc.TcError) as e:
        tc.tc_census_csr_noalloc(tc.TC_NOALLOC_MAX_N + 1, rp, adj, 0, out)
    assert e.value.status == tc.TC_ERR_UNSUPPORTED
    big = 2 * tc.TC_NOALLOC_MAX_DYADS + 2
    adj_big = torch.zeros(big, dtype=torch.int32, device="cuda")
    with pytest.raises(tc.TcError) as e:
        tc.tc_census_csr_noalloc(10, rp, adj_big, big, out)
    assert e.value.status == tc.TC_ERR_UNSUPPORTED


def test_noalloc_checks_the_csr_before_any_census_kernel():
    """Row offsets that do not end at nnz, and a neighbour id outside
    [0, n), are refused; a CSR that lists more canonical dyads than nnz/2
    (not symmetric) is reported as beyond the scratch's capacity.  Every
    call here stays inside the tensors it is given."""
    import torch
    out = torch.zeros(17, dtype=torch.int64, device="cuda")
    dev = lambda a, dt: torch.tensor(a, dtype=dt, device="cuda")
    # row_ptr[n] = 4 but nnz = 2
    rp = dev([0, 2, 4, 4], torch.int64)
    adj = dev([1 << 2 | 1, 2 << 2 | 1, 0 << 2 | 2, 0 << 2 | 2], torch.int32)
    with pytest.raises(tc.TcError) as e:
        tc.tc_census_csr_noalloc(3, rp, adj, 2, out)
    assert e.value.status == tc.TC_ERR_ARG
    # neighbour id 7 in a graph of 3 vertices
    rp = dev([0, 1, 2, 2], torch.int64)
    adj = dev([7 << 2 | 1, 0 << 2 | 2], torch.int32)
    with pytest.raises(tc.TcError) as e:
        tc.tc_census_csr_noalloc(3, rp, adj, 2, out)
    assert e.value.status == tc.TC_ERR_ID_RANGE
    # row 0 lists 1..4, the other rows are empty: 4 canonical dyads, nnz/2 = 2
    rp = dev([0, 4, 4, 4, 4, 4], torch.int64)
    adj = dev([k << 2 | 1 for k in range(1, 5)], torch.int32)
    with pytest.raises(tc.TcError) as e:
        tc.tc_census_csr_noalloc(5, rp, adj, 4, out)
    assert e.value.status == tc.TC_ERR_UNSUPPORTED
    # the scratch is still good for the next call
    arcs = synth.c1()
    rp, adj, nnz = device_csr(arcs)
    tc.tc_census_csr_noalloc(arcs.n, rp, adj, nnz, out)
    assert tc.census_from_device_words(out.cpu().tolist()) == oracle.census(arcs.n, arcs.src, arcs.dst)
