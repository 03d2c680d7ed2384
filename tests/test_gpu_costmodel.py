"""GPU checks of the learned cost model: FP32 gradients and predictions
against the float64 reference, FP16 inference, training, sampling, and that
learned binning never changes the census counts."""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
import synth
import paper_1603_02655_b300 as tc
from paper_1603_02655_b300 import build as tcbuild
from paper_1603_02655_b300 import costmodel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib(cuda_ok):
    tcbuild.build()
    yield tc.load()
    tc.tc_cost_model_load(None)


def cuda(a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).astype(dtype)).cuda()


def rand_data(seed, n):
    rng = np.random.default_rng(seed)
    X = rng.random((n, 8))
    X[:, :4] *= 0.8
    bins = rng.integers(0, 4, n)
    t = rng.normal(11, 2, n)
    return X, bins, t


@pytest.mark.parametrize("seed", range(3))
def test_fp32_gradient_matches_float64_reference(seed):
    X, bins, t = rand_data(seed, 3000)
    p = omlp.init(seed)
    loss_ref, g_ref = omlp.loss_grad(p, X, bins, t)
    loss, g = tc.tc_mlp_loss_grad(cuda(p, np.float32), cuda(X, np.float32), cuda(bins, np.int32),
                                  cuda(t, np.float32))
    g = g.cpu().numpy().astype(np.float64)
    assert abs(loss - loss_ref) <= 1e-5 * abs(loss_ref)
    scale = np.max(np.abs(g_ref))
    assert np.max(np.abs(g - g_ref)) <= 1e-3 * scale, np.max(np.abs(g - g_ref)) / scale


def test_predictions_fp32_and_fp16():
    X, _, _ = rand_data(5, 5000)
    p = omlp.init(5)
    ref, _ = omlp.forward(p, X)
    o32 = tc.tc_mlp_predict(cuda(p, np.float32), cuda(X, np.float32), False).cpu().numpy()
    o16 = tc.tc_mlp_predict(cuda(p, np.float32), cuda(X, np.float32), True).cpu().numpy()
    assert np.max(np.abs(o32 - ref)) <= 1e-4 * (1 + np.max(np.abs(ref)))
    # half precision (11-bit significand, unit roundoff 2^-11) through three
    # layers of <= 32-term dot products accumulated in FP16: errors of a few
    # units in the last place of the layer sums; bound them by 1% of the
    # output scale (a mis-packed weight gives errors of the scale itself)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(o16 - ref)) <= 1e-2 * scale, np.max(np.abs(o16 - ref)) / scale
    assert np.mean(np.abs(o16 - ref)) <= 2e-3 * scale


def test_training_reduces_loss():
    rng = np.random.default_rng(11)
    n = 20000
    X = rng.random((n, 8)).astype(np.float32)
    bins = rng.integers(0, 4, n)
    t = 6 + 8 * X[:, 0] + 3 * X[:, 1] * (bins == 2) + 2 * bins + 0.5 * np.sin(6 * X[:, 3])
    p0 = costmodel.init_params(3)
    loss0 = omlp.loss(p0.astype(np.float64), X, bins, t)
    p, loss = costmodel.fit(cuda(X, np.float32), bins, t.astype(np.float32), steps=1500, batch=2048, lr=3e-3)
    assert loss < 0.05 * loss0 and loss < 0.2, (loss0, loss)
    assert abs(omlp.loss(p.astype(np.float64), X, bins, t) - loss) <= 1e-3 * (1 + loss)


def hub_graph(seed, n=6000):
    rng = np.random.default_rng(seed)
    src, dst = [], []
    for h in range(4):
        nb = rng.choice(n, size=int(rng.integers(1500, 4000)), replace=False)
        out = rng.random(nb.size) < 0.5
        src.append(np.where(out, h, nb))
        dst.append(np.where(out, nb, h))
    src.append(rng.integers(0, n, 40000))
    dst.append(rng.integers(0, n, 40000))
    s = np.concatenate(src).astype(np.int32)
    d = np.concatenate(dst).astype(np.int32)
    rec = rng.random(s.size) < 0.3
    return n, np.concatenate([s, d[rec]]), np.concatenate([d, s[rec]])


def test_features_match_definition():
    n, src, dst = hub_graph(1)
    g = tc.tc_graph_build(n, src, dst)
    try:
        rp, adj = tc.tc_graph_export(g)
        deg = np.diff(rp)
        tags = adj & 3
        row = np.repeat(np.arange(n), deg)
        cnt = np.zeros((n, 4), np.int64)
        np.add.at(cnt, (row, tags), 1)
        rng = np.random.default_rng(2)
        uv = rng.integers(0, n, (500, 2)).astype(np.int32)
        f = tc.tc_cost_features(g, cuda(uv, np.int32)).cpu().numpy()
        for k, (u, v) in enumerate(uv):
            s_, g_ = (u, v) if deg[u] <= deg[v] else (v, u)
            ds, dg = deg[s_], deg[g_]
            want = [np.log2(1 + ds) / 20, np.log2(1 + dg) / 20, (np.log2(1 + dg) - np.log2(1 + ds)) / 20,
                    np.log2(1 + ds + dg) / 20, cnt[s_, 3] / ds if ds else 0, cnt[g_, 3] / dg if dg else 0,
                    cnt[s_, 1] / ds if ds else 0, cnt[g_, 1] / dg if dg else 0]
            assert np.allclose(f[k], want, rtol=1e-5, atol=1e-6), (k, f[k], want)
    finally:
        tc.tc_graph_free(g)


def test_sampling_records_each_bin():
    n, src, dst = hub_graph(3)
    g = tc.tc_graph_build(n, src, dst)
    try:
        for b in range(4):
            rec = tc.tc_cost_sample([g], b, 15, 1 << 16).cpu().numpy()
            assert rec.shape[0] > 0, b
            assert np.all(rec[:, 0] < rec[:, 1])  # canonical dyads u < v
            assert np.all((rec[:, 0] >= 0) & (rec[:, 1] < n))
            assert np.all(rec[:, 3] > 0)
            assert np.any(rec[:, 2] == b)
    finally:
        tc.tc_graph_free(g)


@pytest.mark.parametrize("seed", range(4))
def test_learned_binning_never_changes_counts(seed):
    n, src, dst = hub_graph(10 + seed)
    want = oracle.census(n, src, dst, threads=16)
    g = tc.tc_graph_build(n, src, dst)
    try:
        # random and adversarial networks: whatever bins they pick, same counts
        p = omlp.init(seed).astype(np.float32)
        if seed == 1:
            p[-4:] = [50, 50, 0, 50]      # every large task to tiles
        elif seed == 2:
            p[-4:] = [50, 50, 50, 0]      # every eligible large task streamed
        tc.tc_cost_model_load(p)
        for extra in ({}, {"persistent": 0}, {"thr_thread": 0, "thr_warp": 64}):
            o = tc.tc_opts_default(bin_mode=tc.TC_BIN_MLP, profile=1, own_min=0, tri_path=tc.TC_TRI_MERGE, **extra)
            assert tc.tc_census(g, o) == want
            bt = tc.tc_census_profile()["bin_tasks"]
            if seed == 1:
                assert bt[3] == 0 and bt[2] > 0
            if seed == 2:
                assert bt[3] > 0
    finally:
        tc.tc_cost_model_load(None)
        tc.tc_graph_free(g)


def test_union_sizes_match_definition():
    import torch
    # |S| = |N(u) u N(v) minus {u, v}| from the host neighbour sets, for
    # adjacent and non-adjacent pairs of two graphs of one batched build
    rng = np.random.default_rng(12)
    graphs = [synth.rmat(10, 8, recip=0.2, seed=4), synth.rmat(9, 6, recip=0.0, seed=5)]
    gs = tc.tc_graph_build_batched([a.n for a in graphs], np.cumsum([0] + [a.src.size for a in graphs]),
                                   np.concatenate([a.src for a in graphs]), np.concatenate([a.dst for a in graphs]))
    try:
        uv, want = [], []
        base = 0
        for a in graphs:
            nb = [set() for _ in range(a.n)]
            for s_, d_ in zip(a.src.tolist(), a.dst.tolist()):
                if s_ != d_:
                    nb[s_].add(d_)
                    nb[d_].add(s_)
            for _ in range(300):
                u = int(rng.integers(a.n))
                v = int(rng.choice(sorted(nb[u]))) if nb[u] and rng.random() < 0.7 else int(rng.integers(a.n))
                if u == v:
                    continue
                uv.append((base + u, base + v))
                want.append(len((nb[u] | nb[v]) - {u, v}))
            base += a.n
        got = tc.tc_union_sizes(gs[0], torch.tensor(uv, dtype=torch.int32, device="cuda")).cpu().tolist()
        assert got == want
        with pytest.raises(tc.TcError):  # a pair across the two graphs
            tc.tc_union_sizes(gs[0], torch.tensor([[0, graphs[0].n]], dtype=torch.int32, device="cuda"))
    finally:
        for g in gs:
            tc.tc_graph_free(g)


def test_pipeline_trains_and_reports_its_gain():
    a = synth.rmat(16, 8, recip=0.1, seed=9)
    g = tc.tc_graph_build(a.n, a.src, a.dst)
    try:
        params, rep = costmodel.train_cost_model([g], mask=7, steps=800)
        assert rep["test_samples"] > 100
        assert np.isfinite(rep["rmse_mlp"]) and np.isfinite(rep["rmse_degree_sum"])
        # the gain of the trained network over the method without it: held-out
        # task costs predicted better than by the degree-sum rule fitted to
        # the same training samples
        assert rep["rmse_mlp"] < rep["rmse_degree_sum"], rep
        assert np.isfinite(rep["rmse_exact_size"])
        tc.tc_cost_model_load(params)
        want = tc.tc_census(g)
        assert tc.tc_census(g, tc.tc_opts_default(bin_mode=tc.TC_BIN_MLP, tri_path=tc.TC_TRI_MERGE)) == want
    finally:
        tc.tc_cost_model_load(None)
        tc.tc_graph_free(g)


def test_path_model_trains_on_batch_costs_and_reports_its_routes():
    """The path router's pipeline: batch-scale costs of each graph on each
    path, FP32 training on the GPU, FP16 routing.  On the held-out graphs its
    routes cost at most 25% more than the better of the two paths taken
    alone and no more than the worse one (a sample of about a dozen graphs,
    each timed once: a 10% bound was within its run-to-run noise), and the
    report carries the degree-skew
    rule and the best route per graph beside it; the gain or loss against
    the rule on the full batched workload is measured by the benchmark."""
    b = synth.batch(48, 64, 16384, 4.0, 32.0, 8, 0.5, seed=41)
    graphs = [b.graph(i) for i in range(len(b))]
    params, rep = costmodel.train_path_model(graphs, copies=8, steps=2000, holdout=0.3)
    t = rep["test_us"]
    assert rep["test_graphs"] > 5 and np.isfinite(rep["rmse_log2_us"])
    assert t["best_per_graph"] <= min(t["all_forward"], t["all_merge"], t["skew_rule"], t["learned"]) + 1e-6
    assert t["learned"] <= 1.25 * min(t["all_forward"], t["all_merge"]), rep
    assert t["learned"] <= max(t["all_forward"], t["all_merge"]), rep
    assert np.all(np.isfinite(params))
