"""The warm-start network's GPU kernels (BF16 operands, FP32 accumulation) against the FP64
oracle evaluated with the same BF16-rounded weights, and its training."""
import numpy as np
import pytest

from oracle import mlp as M
from synth import dwell_features, make_patient, mlp_init_params, weights_dirichlet

pytestmark = pytest.mark.gpu


def _bf16_weights(p):
    d = M.unpack(p)
    for k in ("W1", "W2", "W3"):
        d[k] = M.bf16(d[k])
    return M.pack(d)   # biases and w4 stay FP32 on the device too (w4 used in FP32)


def _params(seed):
    p = mlp_init_params(seed).astype(np.float64)
    p += np.random.default_rng(seed).normal(0, 0.02, p.size)   # nonzero biases
    return p.astype(np.float32)


def _batch(seed, R):
    pats = [make_patient(30 + k) for k in range(2)]
    F = np.concatenate([dwell_features(p) for p in pats])
    W = weights_dirichlet(seed, 16)
    rng = np.random.default_rng(seed)
    pairs = np.stack([rng.integers(0, len(F), R), rng.integers(0, len(W), R)], axis=1).astype(np.int32)
    target = rng.uniform(0.0, 4.0, R).astype(np.float32)
    return F, W, pairs, target


def test_predict_matches_oracle(gmco_mod):
    pat = make_patient(7)
    F = dwell_features(pat)
    W = weights_dirichlet(7, 9)
    p = _params(3)
    with gmco_mod.Mlp(p) as net:
        t = net.predict(F, W, t_floor=0.0)
        tf = net.predict(F, W, t_floor=0.5)
    ref, _ = M.forward(_bf16_weights(p), M.dense_inputs(F, W))
    ref = ref.reshape(len(W), len(F))
    err = np.max(np.abs(t - ref)) / np.mean(np.abs(ref))
    print("predict rel err %.2e" % err)
    assert err < 2e-2
    assert np.array_equal(tf, np.maximum(t, 0.5))


@pytest.mark.parametrize("R", [1000, 20000])
def test_gradient_matches_oracle(gmco_mod, R):
    """GPU backward (BF16 activations) vs FP64 backward of the same weights and batch;
    R = 1000 has a ragged last tile, 20000 spans every CTA several times."""
    F, W, pairs, target = _batch(11, R)
    p = _params(5)
    with gmco_mod.Mlp(p) as net:
        loss, g = net.gradient(F, W, pairs, target)
    lref, gref = M.loss_grad(_bf16_weights(p), M.inputs(F, W, pairs), target)
    assert abs(loss / lref - 1.0) < 1e-2, (loss, lref)
    o = 0
    for name, shape in M.SHAPES:
        n = int(np.prod(shape))
        a, b = g[o:o + n], gref[o:o + n]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        print(f"{name}: rel {rel:.2e}")
        assert rel < 2e-2, (name, rel)
        o += n


def test_adam_step_matches_oracle(gmco_mod):
    F, W, pairs, target = _batch(12, 3000)
    p = _params(6)
    lr = 1e-3
    with gmco_mod.Mlp(p) as net:
        _, g = net.gradient(F, W, pairs, target)
        net.train_step(F, W, pairs, target, lr=lr)
        p1 = net.params()
    ref, _, _ = M.adam(p.astype(np.float64), np.zeros(p.size), np.zeros(p.size), g.astype(np.float64), 1, lr)
    assert np.max(np.abs(p1 - ref)) < 1e-6 + 1e-3 * lr


def test_training_reduces_loss(gmco_mod):
    import torch
    F, W, pairs, target = _batch(13, 8192)
    target = (0.5 + np.tanh(M.inputs(F, W, pairs)[:, 0])).astype(np.float32)   # learnable
    dev = [torch.from_numpy(a).cuda() for a in (F, W, pairs, target)]
    with gmco_mod.Mlp(_params(8)) as net:
        first = net.train_step(*dev, lr=2e-3)
        for _ in range(300):
            last = net.train_step(*dev, lr=2e-3)
        launches = net.last_launch_count()
    print("loss %.4f -> %.4f" % (first, last))
    assert last < 0.1 * first
    assert launches > 0
