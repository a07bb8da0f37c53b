"""FP64 reference of the warm-start network.  Test infrastructure only.

The network maps a dwell position's 10 features and a plan's 4 penalty weights to a dwell
time: x0 = [features, log10 max(w, 1e-3)], three hidden layers h = GELU(h W + b) of width
128 with the erf form of GELU, and t = softplus(h_3 . w_4 + b_4).  The training loss is the
mean squared error of t.  Parameters are one flat vector: W_1 (14 x 128, input index
first), b_1, W_2 (128 x 128), b_2, W_3, b_3, w_4 (128), b_4.

Forward and backward are written out layer by layer in float64 (numpy matrix products as
steps), with the erf of scipy.special.  Adam follows Kingma & Ba (2015), Algorithm 1.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

NIN, HID = 14, 128
SHAPES = (("W1", (NIN, HID)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
          ("W3", (HID, HID)), ("b3", (HID,)), ("w4", (HID,)), ("b4", (1,)))
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(params):
    p = np.asarray(params, dtype=np.float64).ravel()
    assert p.size == NPARAM
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_prime(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def softplus(o):
    return np.logaddexp(0.0, o)


def sigmoid(o):
    return 1.0 / (1.0 + np.exp(-o))


def inputs(features, weights, pairs):
    """Rows [R, 14] for pairs (feature row, weight row)."""
    f = np.asarray(features, dtype=np.float64)
    w = np.asarray(weights, dtype=np.float64)
    pr = np.asarray(pairs)
    return np.concatenate([f[pr[:, 0]], np.log10(np.maximum(w[pr[:, 1]], 1e-3))], axis=1)


def dense_inputs(features, weights):
    """Rows of every (plan, dwell) pair, plan-major: row = plan * n_dwell + dwell."""
    nd, P = len(features), len(weights)
    pairs = np.stack([np.tile(np.arange(nd), P), np.repeat(np.arange(P), nd)], axis=1)
    return inputs(features, weights, pairs)


def forward(params, X):
    """Returns t [R] and the intermediate values of the layers."""
    p = unpack(params)
    h0 = np.asarray(X, dtype=np.float64)
    z1 = h0 @ p["W1"] + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = gelu(z2)
    z3 = h2 @ p["W3"] + p["b3"]
    h3 = gelu(z3)
    o = h3 @ p["w4"] + p["b4"][0]
    t = softplus(o)
    return t, dict(h0=h0, z1=z1, h1=h1, z2=z2, h2=h2, z3=z3, h3=h3, o=o)


def loss_grad(params, X, target):
    """Mean squared error of t and its gradient with respect to the flat parameters."""
    p = unpack(params)
    t, c = forward(params, X)
    R = len(t)
    e = t - np.asarray(target, dtype=np.float64)
    loss = float(np.mean(e * e))
    do = 2.0 * e / R * sigmoid(c["o"])                  # dL/do
    g = {"b4": np.array([do.sum()]), "w4": c["h3"].T @ do}
    dz3 = np.outer(do, p["w4"]) * gelu_prime(c["z3"])
    g["W3"], g["b3"] = c["h2"].T @ dz3, dz3.sum(axis=0)
    dz2 = (dz3 @ p["W3"].T) * gelu_prime(c["z2"])
    g["W2"], g["b2"] = c["h1"].T @ dz2, dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"].T) * gelu_prime(c["z1"])
    g["W1"], g["b1"] = c["h0"].T @ dz1, dz1.sum(axis=0)
    return loss, pack(g)


def adam(params, m, v, grad, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (params, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16(x):
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float64."""
    a = np.asarray(x, dtype=np.float32).copy()
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return (u.astype(np.uint32)).view(np.float32).astype(np.float64)
