"""The allocation-free census entry point (tc_census_csr_noalloc).

Callers that may not allocate device memory (their memory manager owns the
GPU, or allocation is forbidden after start-up) pass a CSR they already hold
and get the census computed in the library's fixed scratch area.  This file
is collected last on purpose, and also passes when run alone in a fresh
process.
"""
import numpy as np
import pytest

import synth
import paper_1603_02655_b300 as tc
from paper_1603_02655_b300 import build as tcbuild

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("case", ["c1", "hubs", "empty"])
def test_noalloc_matches_tc_census_on_two_calls_in_a_row(case):
    import torch
    arcs = dict(graphs())[case]
    g = tc.tc_graph_build(arcs.n, arcs.src, arcs.dst)
    try:
        want = tc.tc_census(g)
        rp, adj = tc.tc_graph_export(g)
    finally:
        tc.tc_graph_free(g)
    nnz = int(rp[-1])
    rp_d = torch.from_numpy(rp).cuda()
    adj_d = torch.from_numpy(adj.view(np.int32).copy()).cuda()
    out = torch.zeros(17, dtype=torch.int64, device="cuda")
    for _ in range(2):  # the scratch keeps the last call's contents
        tc.tc_census_csr_noalloc(arcs.n, rp_d, adj_d, nnz, out)
        assert tc.census_from_device_words(out.cpu().tolist()) == want


def test_noalloc_rejects_sizes_beyond_the_maximum():
    import torch
    rp = torch.zeros(tc.TC_NOALLOC_MAX_N + 2, dtype=torch.int64, device="cuda")
    adj = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.zeros(17, dtype=torch.int64, device="cuda")
    with pytest.raises(tc.TcError) as e:
        tc.tc_census_csr_noalloc(tc.TC_NOALLOC_MAX_N + 1, rp, adj, 0, out)
    assert e.value.status == tc.TC_ERR_UNSUPPORTED
    with pytest.raises(tc.TcError) as e:
        tc.tc_census_csr_noalloc(10, rp, adj, 2 * tc.TC_NOALLOC_MAX_DYADS + 2, out)
    assert e.value.status == tc.TC_ERR_UNSUPPORTED
