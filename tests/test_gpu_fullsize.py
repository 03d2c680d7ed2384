"""Full-size parity: the CUDA census of each workload, in the benchmark's
launch configuration, against the census the CPU oracle stored under
tests/golden/ (written by tests/golden/make_golden.py), plus the graph
statistics the oracle recorded with it."""
import json
import os

import pytest

import oracle
import synth
import paper_1603_02655_b300 as tc
from paper_1603_02655_b300 import build as tcbuild

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name):
    path = os.path.join(GOLDEN, f"census_{name}.json")
    if not os.path.exists(path):
        pytest.skip(f"no stored oracle census for {name}")
    return json.load(open(path))


@pytest.fixture(scope="module", autouse=True)
def lib(cuda_ok):
    tcbuild.build()
    return tc.load()


@pytest.mark.parametrize("name", ["c2", "c3", "c5"])
def test_single_graph_workloads_match_oracle(name):
    import torch
    gold = golden(name)
    a = synth.WORKLOADS[name]()
    src = torch.from_numpy(a.src).cuda()
    dst = torch.from_numpy(a.dst).cuda()
    g = tc.tc_graph_build(a.n, src, dst)
    try:
        st = tc.tc_graph_stats(g)
        for k in ("n", "arcs", "dyads", "mutual", "asym", "merged_entries", "max_degree"):
            assert st[k] == gold["stats"][k], k
        c = gold["census"]
        assert sum(c) == a.n * (a.n - 1) * (a.n - 2) // 6
        out = torch.zeros(17, dtype=torch.int64, device="cuda")
        M = tc.TC_TRI_MERGE
        for o in (tc.tc_opts_default(), tc.tc_opts_default(fwd_big=1), tc.tc_opts_default(fwd_big=1 << 30),
                  tc.tc_opts_default(tri_path=M), tc.tc_opts_default(tri_path=M, own_min=0),
                  tc.tc_opts_default(tri_path=M, thr_warp=256, chunk=512, stream_max=256, own_min=1024)):
            tc.tc_census(g, o, out=out)
            torch.cuda.synchronize()
            assert tc.census_from_device_words(out.cpu().tolist()) == c
        assert tc.tc_census(g) == c  # host output path
        # the 64-code census maps onto the golden 16-type census, and the
        # codes agree between the forward and merge paths
        T = oracle.triad_table()
        codes = tc.tc_census_codes(g)
        folded = [0] * 16
        for code, k in enumerate(codes):
            folded[T[code]] += k
        assert folded == c
        assert tc.tc_census_codes(g, tc.tc_opts_default(tri_path=M, own_min=0)) == codes
    finally:
        tc.tc_graph_free(g)


def test_batched_workload_matches_oracle_per_graph():
    """Every one of the 4096 graphs' 16 counts against the oracle's census of
    that graph; the per-type sums and (g+1)-weighted sums are kept as extra
    checks."""
    import torch
    gold = golden("c4")
    b = synth.c4()
    gs = tc.tc_graph_build_batched(b.ns, b.goff, torch.from_numpy(b.src).cuda(), torch.from_numpy(b.dst).cuda())
    try:
        out = torch.zeros(17 * len(gs), dtype=torch.int64, device="cuda")
        plan = tc.tc_plan_create(gs, out)
        tc.tc_plan_run(plan)
        torch.cuda.synchronize()
        tc.tc_plan_free(plan)
        w = out.cpu().tolist()
        census = [tc.census_from_device_words(w[17 * i:17 * i + 17]) for i in range(len(gs))]
        assert len(gold["census"]) == len(census) == 4096
        bad = [i for i, (got, want) in enumerate(zip(census, gold["census"])) if got != want]
        assert not bad, f"{len(bad)} graphs differ, first {bad[:5]}"
        assert [sum(c[t] for c in census) for t in range(16)] == gold["total"]
        assert [sum((i + 1) * c[t] for i, c in enumerate(census)) for t in range(16)] == gold["weighted"]
        for k, v in gold["sample"].items():
            assert census[int(k)] == v["census"], k
            assert tc.tc_graph_stats(gs[int(k)]) == v["stats"], k
    finally:
        for g in gs:
            tc.tc_graph_free(g)
