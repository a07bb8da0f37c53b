"""The annealing engine on the GPU (gmco_solve_sa, the paper's gSA of Sec. 2.2.1) against the
FP64 oracle that draws the same SplitMix64 numbers.

The engines evaluate in different precisions, so a plan's trajectories agree only while no
Metropolis decision lies within rounding of its threshold.  The oracle reports, per plan, how
close its closest decision came (relative to the objectives compared); plans whose closest
decision stayed outside a band many times the form's objective error (FP32 about 1e-7,
bf16x3 about 2e-6) must take the same decisions: the same number of accepted moves and the
same best point and objective."""
import numpy as np
import pytest

from synth import make_class_solution_patient, group_weights, weights_dirichlet

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    p = make_class_solution_patient(6, 12, 0.5, (600, 100, 150, 150), (200, 60, 100, 100))
    W = group_weights(weights_dirichlet(8, 64), p.sid, p.organ).astype(np.float32)
    return p, W


@pytest.mark.parametrize("precision,band,f_tol", [("fp32", 2e-5, 1e-5), ("bf16x3", 5e-5, 3e-5)])
def test_sa_matches_oracle(gmco_mod, oracle_mod, case, precision, band, f_tol):
    p, W = case
    opts = dict(iterations=48, seed=11, T0=1e-2, T_final=1e-5, step0=0.2, step_final=2e-3)
    with gmco_mod.Problem(p.A, p.sid, p.params, precision=precision) as pr:
        out = pr.solve_sa(W, **opts)
    ref = oracle_mod.sa_batch(p.A, p.sid, p.params, W, iters=48, seed=11, T0=1e-2, T_final=1e-5,
                              step0=0.2, step_final=2e-3)
    clear = ref["min_margin"] >= band
    assert clear.sum() >= 8, clear.sum()
    acc, F, T = out["accepts"], out["objectives"], out["T"]
    assert np.array_equal(acc[clear], ref["accepts"][clear])
    assert np.max(np.abs(F[clear] / ref["F"][clear] - 1)) <= f_tol
    scale = ref["T"][clear].max(axis=1, keepdims=True)
    assert np.max(np.abs(T[clear] - ref["T"][clear]) / scale) <= 1e-5
    # every plan: the best objective is no worse than the start (1 s) and moves were taken
    F0 = np.array([oracle_mod.objective(p.A, p.sid, p.params, W[j], np.ones(p.n_dwell),
                                        want_grad=False)[0] for j in range(len(W))])
    assert np.all(F <= F0 * (1 + f_tol)) and np.all((acc > 0) & (acc <= 48))


def test_sa_no_move_device_buffers_and_refusals(gmco_mod, oracle_mod, case):
    import torch
    p, W = case
    t0 = np.random.default_rng(2).uniform(0.5, 6.0, (5, p.n_dwell)).astype(np.float32)
    with gmco_mod.Problem(p.A, p.sid, p.params, precision="fp32") as pr:
        out = pr.solve_sa(torch.from_numpy(W[:5]).cuda(), torch.from_numpy(t0).cuda(),
                          iterations=20, step0=0.0, step_final=0.0)
        assert out["T"].is_cuda
        assert np.array_equal(out["accepts"].cpu().numpy(), np.full(5, 20))
        assert np.allclose(out["T"].cpu().numpy(), t0, rtol=1e-6, atol=0)
        for j in range(5):
            F = oracle_mod.objective(p.A, p.sid, p.params, W[j], np.sqrt(t0[j].astype(np.float64)),
                                     want_grad=False)[0]
            assert abs(float(out["objectives"][j]) / F - 1) <= 1e-5
        zero = pr.solve_sa(W[:2], iterations=0)
        assert np.array_equal(zero["accepts"], [0, 0])
        for kw in (dict(iterations=-1), dict(T0=0.0, T_final=1e-3), dict(step0=float("inf")),
                   dict(iterations=1 << 22)):
            with pytest.raises(gmco_mod.GmcoError) as e:
                pr.solve_sa(W[:2], **kw)
            assert e.value.status == gmco_mod.EINVAL
        with pytest.raises(gmco_mod.GmcoError):
            pr.solve_sa(W[:2], -np.ones((2, p.n_dwell), np.float32), iterations=3)
