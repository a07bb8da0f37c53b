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
    # per element: 2e-2 relative, with a floor of 1e-2 of the mean prediction for the
    # elements near zero (BF16 activations round each layer's inputs to 2^-9)
    bound = 2e-2 * np.abs(ref) + 1e-2 * np.mean(np.abs(ref))
    ratio = np.abs(t - ref) / bound
    w = np.unravel_index(np.argmax(ratio), ratio.shape)
    print("predict: worst element %s, |t - ref| = %.3e, bound %.3e" % (w, abs(t[w] - ref[w]), bound[w]))
    assert np.all(ratio <= 1.0)
    assert np.array_equal(tf, np.maximum(t, 0.5))


def _check_predict(t, ref, label):
    bound = 2e-2 * np.abs(ref) + 1e-2 * np.mean(np.abs(ref))
    ratio = np.abs(t - ref) / bound
    w = np.unravel_index(np.argmax(ratio), ratio.shape)
    print("%s: worst element %s, |t - ref| = %.3e, bound %.3e" % (label, w, abs(t[w] - ref[w]), bound[w]))
    assert np.all(np.isfinite(t)) and np.all(ratio <= 1.0)


@pytest.mark.parametrize("n_cath,n_dwell,n_plans", [
    (18, None, 999),   # 144 dwells x 999 plans = 143856 rows: 1124 tiles, every CTA's
                       # groups loop twice or more, ragged last tile
    (12, None, 1),     # fewer rows than one tile: the CTA's second tile group has no work
    (12, 128, 4),      # whole tiles only
    (12, 1, 1),        # a single row
])
def test_predict_tensor_core_sizes(gmco_mod, n_cath, n_dwell, n_plans):
    """The tcgen05 inference kernel per element against the FP64 forward of the same BF16
    weights, from one row to many persistent-loop rounds, host and device buffers."""
    import torch
    pat = make_patient(40 + n_cath, n_catheters=n_cath)
    F = dwell_features(pat)[:n_dwell]
    W = weights_dirichlet(41, n_plans)
    W[0, 0] = 0.0   # log10 max(w, 1e-3) at its floor
    p = _params(4)
    with gmco_mod.Mlp(p) as net:
        t = net.predict(F, W, t_floor=0.0)
        td = net.predict(torch.from_numpy(F).cuda(), torch.from_numpy(W).cuda(), t_floor=0.0)
        assert net.last_launch_count() == 1
    assert np.array_equal(td.cpu().numpy(), t)
    ref, _ = M.forward(_bf16_weights(p), M.dense_inputs(F, W))
    _check_predict(t, ref.reshape(len(W), len(F)), f"predict {n_plans}x{len(F)}")


def _grad_magnitude(params, X, target):
    """The FP64 backward with every term taken in absolute value: per parameter, the sum of
    the magnitudes of the products whose sum is its gradient.  Rounding the activations and
    deltas to BF16 perturbs each product by a few 2^-9 of its size, so a parameter's error is
    bounded by a small multiple of this sum, whatever the cancellation in the gradient."""
    pr = M.unpack(params)
    t, c = M.forward(params, X)
    R = len(t)
    # e = t - target: its terms' magnitudes, since t carries the forward pass's rounding
    e = np.abs(t) + np.abs(np.asarray(target, dtype=np.float64))
    do = 2.0 * e / R * M.sigmoid(c["o"])
    g = {"b4": np.array([do.sum()]), "w4": np.abs(c["h3"]).T @ do}
    dz3 = np.outer(do, np.abs(pr["w4"])) * np.abs(M.gelu_prime(c["z3"]))
    g["W3"], g["b3"] = np.abs(c["h2"]).T @ dz3, dz3.sum(axis=0)
    dz2 = (dz3 @ np.abs(pr["W3"]).T) * np.abs(M.gelu_prime(c["z2"]))
    g["W2"], g["b2"] = np.abs(c["h1"]).T @ dz2, dz2.sum(axis=0)
    dz1 = (dz2 @ np.abs(pr["W2"]).T) * np.abs(M.gelu_prime(c["z1"]))
    g["W1"], g["b1"] = np.abs(c["h0"]).T @ dz1, dz1.sum(axis=0)
    return M.pack(g)


@pytest.mark.parametrize("R", [1000, 20000])
def test_gradient_matches_oracle(gmco_mod, R):
    """GPU backward (BF16 activations) vs FP64 backward of the same weights and batch;
    R = 1000 has a ragged last tile, 20000 spans every CTA several times."""
    F, W, pairs, target = _batch(11, R)
    p = _params(5)
    with gmco_mod.Mlp(p) as net:
        loss, g = net.gradient(F, W, pairs, target)
    X = M.inputs(F, W, pairs)
    lref, gref = M.loss_grad(_bf16_weights(p), X, target)
    gmag = _grad_magnitude(_bf16_weights(p), X, target)
    assert abs(loss / lref - 1.0) < 1e-2, (loss, lref)
    # every element: |g - g_ref| <= 2e-2 |g_ref| + 1e-2 sum|terms| (see _grad_magnitude;
    # 1e-2 is about five BF16 roundings of 2^-9 along the chain)
    o = 0
    for name, shape in M.SHAPES:
        n = int(np.prod(shape))
        a, b, mg = g[o:o + n], gref[o:o + n], gmag[o:o + n]
        bound = 2e-2 * np.abs(b) + 1e-2 * mg
        ratio = np.abs(a - b) / np.maximum(bound, 1e-30)
        k = int(np.argmax(ratio))
        print(f"{name}: worst element {k}: gpu {a[k]:.4e} ref {b[k]:.4e} |terms| {mg[k]:.3e} "
              f"(error / bound {ratio[k]:.3f}); block rel {np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30):.2e}")
        assert np.all(ratio <= 1.0), (name, k, a[k], b[k], mg[k])
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


def test_checkpoint_resumes_training_bit_for_bit(gmco_mod, tmp_path):
    """save -> load -> train_step gives the parameters of the uninterrupted run, bit for bit
    (the checkpoint holds the FP32 master parameters, both Adam moments and the step count)."""
    F, W, pairs, target = _batch(14, 4096)
    with gmco_mod.Mlp(_params(9)) as net:
        for _ in range(3):
            net.train_step(F, W, pairs, target, lr=1e-3)
        path = tmp_path / "net.gmco"
        net.save(path)
        saved = net.params()
        with gmco_mod.Mlp.load(path) as back:
            assert np.array_equal(back.params(), saved)
            for k in range(4):
                la = net.train_step(F, W, pairs, target, lr=1e-3)
                lb = back.train_step(F, W, pairs, target, lr=1e-3)
                assert la == lb, k
            assert np.array_equal(back.params(), net.params())
    hdr = path.read_bytes().split(b"\n", 2)
    assert hdr[0] == b"GMCO-MLP" and b'"step": 3' in hdr[1]


def test_bad_pairs_refused_without_update(gmco_mod):
    """A pair index out of range is caught by the training kernel before it reads the row: the
    call fails with GMCO_EINVAL and the parameters and the Adam step are unchanged; the next
    valid step runs."""
    F, W, pairs, target = _batch(15, 2000)
    p = _params(10)
    with gmco_mod.Mlp(p) as net:
        for bad in ((0, len(F)), (1, len(W)), (0, -1)):
            pb = pairs.copy()
            pb[777, bad[0]] = bad[1]
            with pytest.raises(gmco_mod.GmcoError) as e:
                net.train_step(F, W, pb, target, lr=1e-3)
            assert e.value.status == gmco_mod.EINVAL
            assert np.array_equal(net.params(), p)
        net.train_step(F, W, pairs, target, lr=1e-3)
        assert not np.array_equal(net.params(), p)
