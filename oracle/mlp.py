"""Float64 reference of the cost-model network -- test infrastructure only.

The task-cost MLP (8 -> 32 -> 32 -> 4, ReLU) and its loss, written from the
textbook definitions: forward pass, loss L = 1/n sum_i 0.5 (o_i[bin_i] -
t_i)^2, and the gradient by the chain rule.  The CUDA library's FP32
training kernels and FP16 inference are checked against it; it is itself
pinned by central finite differences and closed forms (tests/test_mlp_oracle.py).

Parameter layout (flat float64[1476], row = output neuron):
W1[32][8] b1[32] W2[32][32] b2[32] W3[4][32] b3[4].
"""
import numpy as np

IN, H, OUT = 8, 32, 4
SIZES = [("W1", (H, IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (OUT, H)), ("b3", (OUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, k = {}, 0
    for name, shape in SIZES:
        m = int(np.prod(shape))
        out[name] = p[k:k + m].reshape(shape)
        k += m
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def forward(p, X):
    q = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ q["W1"].T + q["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ q["W2"].T + q["b2"]
    h2 = np.maximum(z2, 0.0)
    o = h2 @ q["W3"].T + q["b3"]
    return o, (X, z1, h1, z2, h2)


def loss(p, X, bins, target):
    o, _ = forward(p, X)
    n = len(bins)
    err = o[np.arange(n), np.asarray(bins)] - np.asarray(target, dtype=np.float64)
    return 0.5 * float(np.sum(err * err)) / n


def loss_grad(p, X, bins, target):
    q = unpack(p)
    o, (X, z1, h1, z2, h2) = forward(p, X)
    n = len(bins)
    idx = np.arange(n)
    err = o[idx, np.asarray(bins)] - np.asarray(target, dtype=np.float64)
    d3 = np.zeros_like(o)
    d3[idx, np.asarray(bins)] = err / n
    d2 = (d3 @ q["W3"]) * (z2 > 0)
    d1 = (d2 @ q["W2"]) * (z1 > 0)
    g = {"W3": d3.T @ h2, "b3": d3.sum(0), "W2": d2.T @ h1, "b2": d2.sum(0), "W1": d1.T @ X, "b1": d1.sum(0)}
    return 0.5 * float(np.sum(err * err)) / n, pack(g)


def init(seed=0, scale=1.0):
    """He-style random parameters (normal, std sqrt(2/fan_in)), biases 0."""
    rng = np.random.default_rng(seed)
    d = {"W1": rng.normal(0, np.sqrt(2 / IN), (H, IN)), "b1": np.zeros(H),
         "W2": rng.normal(0, np.sqrt(2 / H), (H, H)), "b2": np.zeros(H),
         "W3": rng.normal(0, np.sqrt(2 / H), (OUT, H)), "b3": np.zeros(OUT)}
    return pack(d) * scale
