"""Training pipeline of the learned task-cost model (calls the C-ABI only).

1. `collect`: instrumented censuses, one per bin with every eligible task
   forced into it, record the cycles of a hashed sample of canonical dyads
   (the same dyads in every bin).  Tiles of a split task are summed per dyad.
2. `features`: the device features of the sampled dyads.
3. `fit`: FP32 Adam training on the GPU (tc_mlp_train) of the 8-32-32-4 MLP
   predicting log2(cycles) per bin.
4. `evaluate`: held-out error of the network against the degree-sum rule of
   the thesis (Sec. 4.3.1: cost |N(u)|+|N(v)|-2), fitted per bin as
   log2(cycles) ~ a + b log2(|N(u)|+|N(v)|) -- the yardstick of the network.
5. `install`: FP16 weights used by census binning (bin_mode = TC_BIN_MLP).
"""
from __future__ import annotations

import numpy as np

from . import (TC_MLP_NPARAM, tc_cost_features, tc_cost_model_load, tc_cost_sample, tc_graph_stats,
               tc_mlp_predict, tc_mlp_train, tc_union_sizes)

BINS = 4


def init_params(seed: int = 0) -> np.ndarray:
    """He-initialised parameters (float32), output bias 10 (~ log2 of a few
    thousand cycles) so training starts near the data."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, np.sqrt(2 / 8), (32, 8)), np.zeros(32), rng.normal(0, np.sqrt(2 / 32), (32, 32)),
             np.zeros(32), rng.normal(0, np.sqrt(2 / 32), (4, 32)), np.full(4, 10.0)]
    p = np.concatenate([x.reshape(-1) for x in parts]).astype(np.float32)
    assert p.size == TC_MLP_NPARAM
    return p


def collect(gs, mask: int = 63, cap: int = 1 << 21, bins=range(BINS), stream=None):
    """Sampled task costs: (uv int32[n,2], bin int32[n], log2 cycles float32[n])."""
    uv_all, bin_all, tgt_all = [], [], []
    for b in bins:
        rec = tc_cost_sample(gs, b, mask, cap, stream).cpu().numpy()
        if rec.size == 0:
            continue
        rec = rec[rec[:, 2] == b]  # only tasks that ran in the forced bin
        key = rec[:, 0].astype(np.int64) << 32 | rec[:, 1].astype(np.int64)
        uniq, inv = np.unique(key, return_inverse=True)
        cyc = np.zeros(uniq.size, dtype=np.float64)
        np.add.at(cyc, inv, rec[:, 3].astype(np.float64))
        uv = np.stack([(uniq >> 32).astype(np.int32), (uniq & 0xffffffff).astype(np.int32)], axis=1)
        uv_all.append(uv)
        bin_all.append(np.full(uniq.size, b, dtype=np.int32))
        tgt_all.append(np.log2(np.maximum(cyc, 1.0)).astype(np.float32))
    if not uv_all:
        return (np.zeros((0, 2), np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32))
    return np.concatenate(uv_all), np.concatenate(bin_all), np.concatenate(tgt_all)


def features(g, uv: np.ndarray, stream=None):
    import torch
    return tc_cost_features(g, torch.from_numpy(np.ascontiguousarray(uv)).cuda(), stream)


def fit(feat, bins: np.ndarray, target: np.ndarray, steps: int = 3000, batch: int = 4096, lr: float = 3e-3,
        seed: int = 1, params: np.ndarray | None = None, stream=None):
    """Train on the GPU; returns (params float32[1476], final loss)."""
    import torch
    p = torch.from_numpy(init_params(seed) if params is None else params.astype(np.float32)).cuda()
    b = torch.from_numpy(bins.astype(np.int32)).cuda()
    t = torch.from_numpy(target.astype(np.float32)).cuda()
    loss = tc_mlp_train(p, feat, b, t, steps, min(batch, feat.shape[0]), lr, seed, stream)
    return p.cpu().numpy(), loss


def union_sizes(g, uv: np.ndarray, stream=None) -> np.ndarray:
    """|S| of each sampled task (the exact cost of Sec. 4.3.1), from the GPU."""
    import torch
    return tc_union_sizes(g, torch.from_numpy(np.ascontiguousarray(uv)).cuda(), stream).cpu().numpy()


def evaluate(params: np.ndarray, feat, bins: np.ndarray, target: np.ndarray, train_mask: np.ndarray,
             s_exact: np.ndarray | None = None) -> dict:
    """Held-out RMSE (in log2 cycles) of the network (FP16 inference, as used
    by binning), of the degree-sum rule fitted per bin on the training part,
    and (given |S| per task) of the same fit on the exact cost |S|: the
    ceiling of a one-number cost rule."""
    import torch
    p = torch.from_numpy(params.astype(np.float32)).cuda()
    pred = tc_mlp_predict(p, feat, True).cpu().numpy()
    f = feat.cpu().numpy()
    # |N(u)|+|N(v)| from feature 3 = log2(1 + d_s + d_g) / 20
    L = np.exp2(f[:, 3] * 20.0) - 1.0
    test = ~train_mask
    out = {"samples": int(bins.size), "test_samples": int(test.sum()), "per_bin": {}}
    se_mlp = se_heur = se_exact = 0.0
    for b in range(BINS):
        tr = train_mask & (bins == b)
        te = test & (bins == b)
        if tr.sum() < 2 or te.sum() == 0:
            continue
        A = np.stack([np.ones(tr.sum()), np.log2(L[tr])], axis=1)
        coef, *_ = np.linalg.lstsq(A, target[tr], rcond=None)
        h = coef[0] + coef[1] * np.log2(L[te])
        e_mlp = pred[te, b] - target[te]
        e_heur = h - target[te]
        se_mlp += float(np.sum(e_mlp ** 2))
        se_heur += float(np.sum(e_heur ** 2))
        if s_exact is not None:
            ls = np.log2(1.0 + s_exact.astype(np.float64))
            cx, *_ = np.linalg.lstsq(np.stack([np.ones(tr.sum()), ls[tr]], axis=1), target[tr], rcond=None)
            se_exact += float(np.sum((cx[0] + cx[1] * ls[te] - target[te]) ** 2))
        out["per_bin"][b] = {"n_test": int(te.sum()), "rmse_mlp": float(np.sqrt(np.mean(e_mlp ** 2))),
                             "rmse_degree_sum": float(np.sqrt(np.mean(e_heur ** 2)))}
    nt = max(1, int(test.sum()))
    out["rmse_mlp"] = float(np.sqrt(se_mlp / nt))
    out["rmse_degree_sum"] = float(np.sqrt(se_heur / nt))
    if s_exact is not None:
        out["rmse_exact_size"] = float(np.sqrt(se_exact / nt))
    return out


def install(params) -> None:
    tc_cost_model_load(params)


def train_cost_model(gs, mask: int = 63, steps: int = 3000, batch: int = 4096, lr: float = 3e-3, seed: int = 1,
                     holdout: float = 0.2, stream=None):
    """Collect, train, evaluate; returns (params, report).  Does not install."""
    uv, bins, target = collect(gs, mask, stream=stream)
    if bins.size < 16:
        raise ValueError("too few sampled tasks to train the cost model")
    feat = features(gs[0], uv, stream)
    rng = np.random.default_rng(seed)
    train_mask = rng.random(bins.size) >= holdout
    import torch
    idx = torch.from_numpy(np.nonzero(train_mask)[0]).cuda()
    params, loss = fit(feat[idx].contiguous(), bins[train_mask], target[train_mask], steps, batch, lr, seed,
                       stream=stream)
    rep = evaluate(params, feat, bins, target, train_mask, union_sizes(gs[0], uv, stream))
    rep["train_loss"] = loss
    rep["graph_stats"] = [tc_graph_stats(g) for g in gs[:4]]
    return params, rep


# ------------------------------------------------------------ path routing
# The same network, trained on graph-level features (tc_path_features) to
# predict log2 of a graph's census time on each path (output 0 forward,
# 1 merge); TC_TRI_AUTO sends each graph to the cheaper prediction.  The
# yardstick is the degree-skew rule (forward when the largest degree is at
# least 8x the mean degree), the router without a model.

def call_costs(gs, reps: int = 3, stream=None) -> np.ndarray:
    """Single-call census time (microseconds, CUDA events, best of `reps`
    after one warm-up) of each graph on the forward and on the merge path:
    float[G, 2].  (Dominated by the fixed cost per call for small graphs; the
    router is trained on `batch_costs` instead.)"""
    import torch
    from . import TC_TRI_FORWARD, TC_TRI_MERGE, tc_census, tc_opts_default
    st = torch.cuda.current_stream() if stream is None else stream
    out = torch.zeros(17, dtype=torch.int64, device="cuda")
    costs = np.zeros((len(gs), 2))
    for k, path in enumerate((TC_TRI_FORWARD, TC_TRI_MERGE)):
        o = tc_opts_default(tri_path=path)
        for i, g in enumerate(gs):
            best = float("inf")
            for r in range(reps + 1):
                a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(st)
                tc_census(g, o, out=out, stream=st)
                c.record(st)
                torch.cuda.synchronize()
                if r > 0:
                    best = min(best, a.elapsed_time(c) * 1e3)
            costs[i, k] = best
    return costs


def skew_rule(feat: np.ndarray) -> np.ndarray:
    """The router without a model: 1 (merge) unless max degree >= 8 x mean
    degree (feature 4 = log2(max/mean) / 8)."""
    return (feat[:, 4] * 8.0 < 3.0).astype(np.int32)


def batch_costs(graphs, copies: int = 32, reps: int = 3, stream=None) -> tuple[np.ndarray, np.ndarray]:
    """A graph's cost inside a batched census (microseconds) on each path:
    each graph (objects with n, src, dst) is built `copies` times into one
    batched build, and its cost is (time of the census of all copies - time
    of one copy) / (copies - 1), so the census's fixed cost per call
    (launches, scans, the fold) cancels and the kernels run at batch scale.
    Returns (features float32[G, 8], costs float[G, 2])."""
    import torch
    from . import (TC_TRI_FORWARD, TC_TRI_MERGE, tc_census_batched, tc_graph_build_batched, tc_graph_free,
                   tc_opts_default, tc_path_features)
    st = torch.cuda.current_stream() if stream is None else stream
    out = torch.zeros(17 * copies, dtype=torch.int64, device="cuda")

    def best(sub, o):
        t = float("inf")
        for r in range(reps + 1):
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            tc_census_batched(sub, o, out=out[:17 * len(sub)], stream=st)
            c.record(st)
            torch.cuda.synchronize()
            if r > 0:
                t = min(t, a.elapsed_time(c) * 1e3)
        return t

    feats, costs = [], []
    for a in graphs:
        m = int(a.src.size)
        src = torch.from_numpy(np.tile(np.asarray(a.src, np.int32), copies)).cuda()
        dst = torch.from_numpy(np.tile(np.asarray(a.dst, np.int32), copies)).cuda()
        gs = tc_graph_build_batched(np.full(copies, a.n, np.int32), np.arange(copies + 1, dtype=np.int64) * m,
                                    src, dst)
        try:
            feats.append(tc_path_features(gs[:1])[0])
            row = []
            for path in (TC_TRI_FORWARD, TC_TRI_MERGE):
                o = tc_opts_default(tri_path=path)
                row.append(max((best(gs, o) - best(gs[:1], o)) / (copies - 1), 1.0))
            costs.append(row)
        finally:
            for g in gs:
                tc_graph_free(g)
    return np.array(feats, np.float32).reshape(-1, 8), np.array(costs, np.float64).reshape(-1, 2)


def train_path_model(graphs, copies: int = 32, steps: int = 4000, lr: float = 3e-3, seed: int = 1,
                     holdout: float = 0.25, stream=None):
    """Measure (`batch_costs`), train (FP32 kernels) and evaluate the path
    model on a list of graphs (objects with n, src, dst); returns (params,
    report).  Does not install.  The report compares, on the held-out
    graphs, the summed batch costs of the learned routes with the
    degree-skew rule's, each path alone, and the best route per graph."""
    import torch
    feat, costs = batch_costs(graphs, copies, stream=stream)
    G = costs.shape[0]
    rng = np.random.default_rng(seed)
    train = rng.random(G) >= holdout
    # one sample per graph and path: the output of that path is trained
    f2 = np.repeat(feat, 2, axis=0)
    b2 = np.tile(np.array([0, 1], np.int32), G)
    t2 = np.log2(np.maximum(costs.reshape(-1), 1.0)).astype(np.float32)
    m2 = np.repeat(train, 2)
    params, loss = fit(torch.from_numpy(f2[m2]).cuda(), b2[m2], t2[m2], steps, 4096, lr, seed, stream=stream)
    p = torch.from_numpy(params).cuda()
    pred = tc_mlp_predict(p, torch.from_numpy(feat).cuda(), True).cpu().numpy()[:, :2]
    learned = (pred[:, 1] < pred[:, 0]).astype(np.int32)
    rule = skew_rule(feat)
    best = np.argmin(costs, axis=1)
    test = ~train

    def cost(route, mask):
        return float(costs[np.arange(G)[mask], route[mask]].sum())

    rep = {"graphs": G, "test_graphs": int(test.sum()), "copies": copies, "train_loss": loss,
           "rmse_log2_us": float(np.sqrt(np.mean((pred[test] - np.log2(np.maximum(costs[test], 1.0))) ** 2))),
           "test_us": {"all_forward": cost(np.zeros(G, np.int32), test), "all_merge": cost(np.ones(G, np.int32), test),
                       "skew_rule": cost(rule, test), "learned": cost(learned, test),
                       "best_per_graph": cost(best, test)},
           "test_agreement_with_best": {"learned": float(np.mean(learned[test] == best[test])),
                                        "skew_rule": float(np.mean(rule[test] == best[test]))}}
    return params, rep
