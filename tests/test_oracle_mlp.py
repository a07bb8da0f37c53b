"""Pins of the FP64 warm-start network oracle against facts outside itself: central finite
differences of its loss, closed forms of a network whose hidden weights are zero, values of
the standard normal CDF, Adam's first step (Kingma & Ba 2015: |step| = lr for every
parameter with a nonzero gradient) and bfloat16 rounding of exactly representable and tie
values."""
import math

import numpy as np
import pytest

from oracle import mlp as M
from synth import make_patient, dwell_features, mlp_init_params, weights_dirichlet


def _batch(seed=0, R=24):
    pat = make_patient(3)
    F = dwell_features(pat)
    W = weights_dirichlet(seed, 6)
    rng = np.random.default_rng(seed)
    pairs = np.stack([rng.integers(0, len(F), R), rng.integers(0, len(W), R)], axis=1)
    X = M.inputs(F, W, pairs)
    target = rng.uniform(0.0, 3.0, R)
    return X, target


def test_layout_matches_documented_count():
    assert M.NPARAM == 14 * 128 + 128 + 2 * (128 * 128 + 128) + 128 + 1 == 35073
    p = mlp_init_params(0)
    assert p.shape == (M.NPARAM,) and np.all(np.isfinite(p))
    assert abs(M.softplus(M.unpack(p)["b4"][0]) - 1.0) < 1e-6   # softplus(b4) = 1 s


def test_gelu_is_z_times_normal_cdf():
    # Phi(1) = 0.8413447460685429, Phi(-1) = 0.15865525393145707, Phi(2) = 0.9772498680518208
    z = np.array([1.0, -1.0, 2.0, 0.0])
    want = z * np.array([0.8413447460685429, 0.15865525393145707, 0.9772498680518208, 0.5])
    assert np.allclose(M.gelu(z), want, rtol=0, atol=1e-15)
    assert M.gelu_prime(np.array([0.0]))[0] == 0.5
    # derivative against a central difference of the function
    zz = np.linspace(-4, 4, 17)
    h = 1e-6
    fd = (M.gelu(zz + h) - M.gelu(zz - h)) / (2 * h)
    assert np.max(np.abs(fd - M.gelu_prime(zz))) < 1e-8
    assert abs(M.softplus(np.array([0.0]))[0] - math.log(2.0)) < 1e-15


def test_gradient_against_central_differences():
    X, target = _batch()
    p = mlp_init_params(1).astype(np.float64)
    rng = np.random.default_rng(2)
    p = p + rng.normal(0, 0.05, p.size)   # generic point: nonzero biases
    _, g = M.loss_grad(p, X, target)
    blocks, o = {}, 0
    for name, shape in M.SHAPES:
        n = int(np.prod(shape))
        blocks[name] = (o, n)
        o += n
    for name, (o, n) in blocks.items():
        for i in rng.choice(n, size=min(n, 6), replace=False):
            k = o + i
            h = 1e-6 * max(1.0, abs(p[k]))
            pp, pm = p.copy(), p.copy()
            pp[k] += h
            pm[k] -= h
            fd = (M.loss_grad(pp, X, target)[0] - M.loss_grad(pm, X, target)[0]) / (2 * h)
            assert abs(fd - g[k]) <= 1e-6 * max(1e-3, np.max(np.abs(g))), (name, i, fd, g[k])


def test_zero_hidden_weights_closed_form():
    X, target = _batch(R=10)
    d = M.unpack(mlp_init_params(4))
    d = {k: v.copy() for k, v in d.items()}
    for k in ("W1", "W2", "W3"):
        d[k][:] = 0.0
    d["b1"][:] = 0.3
    d["b2"][:] = -0.2
    d["b3"][:] = 0.7
    p = M.pack(d)
    t, _ = M.forward(p, X)
    o = d["w4"] @ np.full(128, 0.7 * 0.5 * (1 + math.erf(0.7 / math.sqrt(2)))) + d["b4"][0]
    y = math.log1p(math.exp(o))
    assert np.allclose(t, y, rtol=1e-14)
    loss, g = M.loss_grad(p, X, target)
    assert abs(loss - np.mean((y - target) ** 2)) < 1e-13
    s = 1.0 / (1.0 + math.exp(-o))
    assert abs(g[-1] - np.mean(2 * (y - target)) * s) < 1e-13          # b4
    h3 = 0.7 * 0.5 * (1 + math.erf(0.7 / math.sqrt(2)))
    assert np.allclose(g[-129:-1], np.mean(2 * (y - target)) * s * h3, rtol=1e-12)   # w4


def test_adam_first_step_moves_by_lr():
    rng = np.random.default_rng(5)
    p = rng.normal(size=50)
    g = rng.normal(size=50)
    g[3] = 0.0
    p1, m, v = M.adam(p, np.zeros(50), np.zeros(50), g, 1, lr=1e-3)
    step = p - p1
    mask = g != 0
    assert np.allclose(np.abs(step[mask]), 1e-3, rtol=1e-6)
    assert np.all(np.sign(step[mask]) == np.sign(g[mask]))
    assert step[3] == 0.0


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.0e-5], dtype=np.float32)
    r = M.bf16(x)
    assert r[0] == 1.0 and r[3] == -2.5
    assert r[1] == 1.0                      # tie: to even
    assert r[2] == 1.0 + 2 ** -7            # nearest (0.75 of a step above 1)
    assert abs(r[4] / 3.0e-5 - 1) < 2 ** -8


def test_inputs_floor_log_weights():
    F = np.arange(20, dtype=np.float32).reshape(2, 10)
    W = np.array([[10.0, 1.0, 0.1, 0.0]], dtype=np.float32)
    X = M.inputs(F, W, np.array([[1, 0]]))
    assert np.array_equal(X[0, :10], F[1])
    assert np.allclose(X[0, 10:], [1.0, 0.0, -1.0, -3.0])
