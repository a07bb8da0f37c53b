"""Dose rate matrix on the GPU (gmco_dose_rate_matrix, step (i) of the planning flow) against
the FP64 oracle of the same point-source model.

FP32 evaluation: the constant K, the distance (one square root), g(r), r^2 and one division
each round once, so the relative error stays within about 8 units of 2^-24 (5e-7); bound 2e-6.
"""
import numpy as np
import pytest

from synth import make_patient

pytestmark = pytest.mark.gpu


def test_rates_match_oracle_host_and_device(gmco_mod, oracle_mod):
    p = make_patient(21, 20, 0.2, (1500, 200, 400, 400), 1.3)   # 460 dwells
    pts, dws = p.points.astype(np.float32), p.dwells.astype(np.float32)   # the library's inputs
    ref = oracle_mod.dose_rate(pts, dws)
    A = gmco_mod.dose_rate_matrix(pts, dws)
    assert A.shape == ref.shape and A.dtype == np.float32
    assert np.max(np.abs(A - ref) / ref) <= 2e-6
    import torch
    At = gmco_mod.dose_rate_matrix(torch.from_numpy(pts).cuda(), torch.from_numpy(dws).cuda())
    torch.cuda.synchronize()
    assert At.is_cuda and np.array_equal(At.cpu().numpy(), A)


def test_clamp_ragged_and_refusals(gmco_mod, oracle_mod):
    rng = np.random.default_rng(5)
    dw = rng.uniform(-2, 2, (1, 3))
    # points on, inside and outside the 0.1 cm clamp, one point row per block and a single dwell
    pts = np.concatenate([dw, dw + [0.05, 0, 0], dw + [0, 0.1, 0],
                          rng.uniform(-3, 3, (2999, 3))]).astype(np.float32)
    dw = dw.astype(np.float32)
    A = gmco_mod.dose_rate_matrix(pts, dw)
    ref = oracle_mod.dose_rate(pts, dw)
    assert A[0, 0] == A[1, 0]                            # both inside the clamp
    assert A[2, 0] == pytest.approx(A[0, 0], rel=1e-6)   # on its edge, up to FP32 rounding of r
    assert np.max(np.abs(A - ref) / ref) <= 2e-6
    # 1024 dwells (the largest problem), 3 points
    dw2 = rng.uniform(-2, 2, (1024, 3)).astype(np.float32)
    A2 = gmco_mod.dose_rate_matrix(pts[:3], dw2)
    assert np.max(np.abs(A2 - oracle_mod.dose_rate(pts[:3], dw2)) / oracle_mod.dose_rate(pts[:3], dw2)) <= 2e-6
    for bad_pts, bad_dw in (([[30.0, 0, 0]], [[0.0, 0, 0]]),       # g(r) < 0 beyond ~23.6 cm
                            ([[np.nan, 0, 0]], [[0.0, 0, 0]]),
                            (np.zeros((2, 3)), np.zeros((1025, 3)))):
        with pytest.raises(gmco_mod.GmcoError) as e:
            gmco_mod.dose_rate_matrix(np.array(bad_pts, np.float32), np.array(bad_dw, np.float32))
        assert e.value.status == gmco_mod.EINVAL
    with pytest.raises(gmco_mod.GmcoError):
        gmco_mod.dose_rate_matrix(pts, dw, source=gmco_mod.default_source(r_min=0.0))


def test_problem_from_device_rates(gmco_mod, oracle_mod):
    """A problem created straight from the device matrix evaluates as the oracle does on the
    same (FP32) matrix."""
    import torch
    p = make_patient(4, 12, 0.5, (700, 100, 150, 150))
    At = gmco_mod.dose_rate_matrix(torch.from_numpy(p.points.astype(np.float32)).cuda(),
                                   torch.from_numpy(p.dwells.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    A = At.cpu().numpy()
    W = np.full((3, 4), 1.0, np.float32)
    X = np.random.default_rng(4).uniform(0.5, 1.5, (3, p.n_dwell)).astype(np.float32)
    with gmco_mod.Problem(At, p.sid, p.params, precision="fp32") as pr:
        out = pr.evaluate(W, X, objectives=True, grad=False, dose=True)
    for j in range(3):
        F, _, d, _ = oracle_mod.objective(A, p.sid, p.params, W[j], X[j])
        assert np.max(np.abs(out["dose"][j] - d) / d) <= 1e-5
        assert abs(out["objectives"][j] / F - 1.0) <= 2e-5
