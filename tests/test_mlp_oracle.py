"""Pins for the float64 cost-model reference (no GPU): its gradient against
central finite differences, and closed forms of the forward pass and loss."""
import numpy as np
import pytest

from oracle import mlp


def data(seed, n=64):
    rng = np.random.default_rng(seed)
    X = rng.random((n, mlp.IN))
    bins = rng.integers(0, mlp.OUT, n)
    t = rng.normal(10, 3, n)
    return X, bins, t


@pytest.mark.parametrize("seed", range(3))
def test_gradient_matches_central_differences(seed):
    p = mlp.init(seed)
    X, bins, t = data(seed)
    _, g = mlp.loss_grad(p, X, bins, t)
    rng = np.random.default_rng(100 + seed)
    for k in rng.choice(mlp.NPARAM, 80, replace=False):
        h = 1e-6
        e = np.zeros(mlp.NPARAM)
        e[k] = h
        num = (mlp.loss(p + e, X, bins, t) - mlp.loss(p - e, X, bins, t)) / (2 * h)
        assert abs(num - g[k]) <= 1e-6 * max(1.0, abs(num)), (k, num, g[k])


def test_closed_forms():
    X, bins, t = data(7, 16)
    # all weights zero: the output is the last bias, the loss a plain mean
    d = {k: np.zeros(s) for k, s in mlp.SIZES}
    d["b3"] = np.array([1.0, 2.0, 3.0, 4.0])
    p = mlp.pack(d)
    o, _ = mlp.forward(p, X)
    assert np.allclose(o, d["b3"])
    pred = d["b3"][bins]
    assert np.isclose(mlp.loss(p, X, bins, t), 0.5 * np.mean((pred - t) ** 2))
    _, g = mlp.loss_grad(p, X, bins, t)
    gd = mlp.unpack(g)
    for k in range(4):  # d/db3_k = mean over samples of bin k of (pred - t)
        sel = bins == k
        assert np.isclose(gd["b3"][k], np.sum(pred[sel] - t[sel]) / len(bins))
    assert np.allclose(gd["W1"], 0) and np.allclose(gd["W2"], 0)
    # identity-like positive path: linear network on positive inputs
    d = {k: np.zeros(s) for k, s in mlp.SIZES}
    d["W1"][0, 0] = 2.0
    d["W2"][0, 0] = 3.0
    d["W3"][:, 0] = 0.5
    p = mlp.pack(d)
    o, _ = mlp.forward(p, X)
    assert np.allclose(o, 3.0 * X[:, :1])
    assert mlp.NPARAM == 1476
