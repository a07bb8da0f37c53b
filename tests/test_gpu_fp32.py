"""FP32 form on the GPU vs the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from synth import make_patient, workload
from tests.conftest import read_fstar

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small():
    p, W, _ = workload("prostate-2k-8plans")
    return p, W


@pytest.fixture(scope="module")
def prob_fp32(gmco_mod, small):
    p, _ = small
    pr = gmco_mod.Problem(p.A, p.sid, p.params, precision="fp32")
    yield pr
    pr.close()


def _ragged(seed=4):
    """n_pnt = 1037 (not a tile multiple), n_dwell = 45, 70 plans."""
    p = make_patient(seed, 12, 0.5, (700, 100, 150, 150))
    rng = np.random.default_rng(seed)
    rows = np.sort(rng.permutation(p.n_pnt)[:1037])
    A = np.ascontiguousarray(p.A[rows][:, :45])
    sid = p.sid[rows]
    W = (10.0 ** rng.uniform(-1, 1, (70, 4))).astype(np.float32)
    X = rng.uniform(0.3, 2.0, (70, 45)).astype(np.float32)
    return A, sid, p.params, W, X


def _check_eval(oracle_mod, A, sid, prm, W, X, out, tol=1e-5):
    for j in range(W.shape[0]):
        F, g, d, _ = oracle_mod.objective(A, sid, prm, W[j], X[j])
        assert np.max(np.abs(out["dose"][j] - d) / np.maximum(np.abs(d), 1e-30)) <= tol
        assert abs(out["objectives"][j] - F) <= tol * F
        assert np.max(np.abs(out["grad"][j] - g)) <= tol * np.max(np.abs(g))


def test_evaluate_parity_small(gmco_mod, oracle_mod, small, prob_fp32):
    p, W = small
    X = np.random.default_rng(0).uniform(0.5, 1.5, (8, p.n_dwell)).astype(np.float32)
    out = prob_fp32.evaluate(W, X, objectives=True, grad=True, dose=True, dvh=True)
    _check_eval(oracle_mod, p.A, p.sid, p.params, W, X, out)


def test_evaluate_parity_ragged(gmco_mod, oracle_mod):
    A, sid, prm, W, X = _ragged()
    with gmco_mod.Problem(A, sid, prm) as pr:
        out = pr.evaluate(W, X, objectives=True, grad=True, dose=True)
    _check_eval(oracle_mod, A, sid, prm, W, X, out)


def test_dvh_exact_on_same_doses(gmco_mod, oracle_mod, small, prob_fp32):
    p, _ = small
    rng = np.random.default_rng(2)
    D = rng.uniform(5.0, 25.0, (16, p.n_pnt)).astype(np.float32)
    D[3, p.sid == 0] = 15.0                 # ties at the threshold count as receiving it
    got = prob_fp32.dvh_from_dose(D)
    for j in range(16):
        ref = oracle_mod.dvh(D[j], p.sid, 4, 15.0).astype(np.float32)
        assert np.array_equal(got[j], ref), (j, got[j], ref)


def test_solve_reaches_exact_optimum(gmco_mod, oracle_mod, small, prob_fp32):
    p, W = small
    fstar = read_fstar("prostate-2k-8plans")
    out = prob_fp32.solve_batch(W, max_iters=20000, tol=1e-10)
    gaps = []
    for j in range(8):
        F = oracle_mod.objective(p.A, p.sid, p.params, W[j], np.sqrt(out["T"][j]))[0]
        assert abs(out["objectives"][j] / F - 1.0) <= 1e-5    # reported F is the plan's F
        gaps.append(F / fstar[j] - 1.0)
    print("fp32 gaps", gaps, out["iters"], out["status"])
    assert min(gaps) >= -1e-9                 # nothing beats the exact optimum
    assert sum(g <= 1e-4 for g in gaps) >= 7  # the relative-change rule can stop one early
    assert np.all(out["T"] >= 0)


def test_dvh_of_solution_matches_oracle_at_same_T(gmco_mod, oracle_mod, small, prob_fp32):
    p, W = small
    out = prob_fp32.solve_batch(W, max_iters=300, tol=0.0)
    for j in range(8):
        d = oracle_mod.dose(p.A, out["T"][j])
        ref = oracle_mod.dvh(d, p.sid, 4, 15.0)
        assert abs(out["dvh"][j][0] - ref[0]) <= 0.5      # V100, percentage points
        assert abs(out["dvh"][j][1] - ref[1]) <= 0.5      # D90, % of Rx
        F = oracle_mod.objective(p.A, p.sid, p.params, W[j], np.sqrt(out["T"][j]))[0]
        assert abs(out["objectives"][j] / F - 1.0) <= 1e-5


def test_first_iterations_follow_oracle(gmco_mod, oracle_mod, small, prob_fp32):
    p, W = small
    for k in (1, 2):
        out = prob_fp32.solve_batch(W, max_iters=k, tol=0.0)
        for j in range(8):
            r = oracle_mod.lbfgs(p.A, p.sid, p.params, W[j], None, max_iters=k, tol=0.0)
            assert out["iters"][j] == r["iters"] == k
            assert abs(out["objectives"][j] / r["F"] - 1.0) <= 1e-5
            assert np.allclose(out["T"][j], r["t"], rtol=1e-4, atol=1e-6)



def test_evaluation_budget_follows_oracle(gmco_mod, oracle_mod, small):
    """max_evals: every plan stops after the same evaluations and iterations as the oracle with
    the same budget, at the same point."""
    p, W = small
    for cap in (1, 5):
        with gmco_mod.Problem(p.A, p.sid, p.params, precision="fp32", max_evals=cap) as pr:
            out = pr.solve_batch(W, max_iters=100, tol=0.0)
        for j in range(8):
            r = oracle_mod.lbfgs(p.A, p.sid, p.params, W[j], None, max_iters=100, tol=0.0,
                                 max_evals=cap)
            assert out["status"][j] == r["status"] == oracle_mod.MAXITER
            assert out["iters"][j] == r["iters"]
            assert abs(out["objectives"][j] / r["F"] - 1.0) <= 1e-5
            assert np.allclose(out["T"][j], r["t"], rtol=1e-4, atol=1e-6)

def test_zero_objective_start(gmco_mod, small):
    p, W = small
    d0 = p.A.astype(np.float64) @ np.ones(p.n_dwell)
    prm = p.params.copy()
    prm[0, 1] = d0[p.sid == 0].min() - 0.1
    for s in (1, 2, 3):
        prm[s, 2] = d0[p.sid == s].max() + 0.1
    with gmco_mod.Problem(p.A, p.sid, prm) as pr:
        out = pr.solve_batch(W, max_iters=50, tol=1e-6)
    assert np.all(out["iters"] == 0) and np.all(out["status"] == 0)
    assert np.all(out["objectives"] == 0.0) and np.all(out["T"] == 1.0)


def test_max_iters_zero(gmco_mod, small, prob_fp32):
    p, W = small
    t0 = np.full((8, p.n_dwell), 2.25, np.float32)
    out = prob_fp32.solve_batch(W, t0=t0, max_iters=0, tol=1e-6)
    assert np.all(out["status"] == 1) and np.all(out["iters"] == 0)
    assert np.array_equal(out["T"], t0)


def test_batch_invariance(gmco_mod, small, prob_fp32):
    p, W = small
    full = prob_fp32.solve_batch(W, max_iters=150, tol=1e-7)
    for j in (0, 5):
        one = prob_fp32.solve_batch(W[j:j + 1], max_iters=150, tol=1e-7)
        assert np.array_equal(one["T"][0], full["T"][j])
        assert one["objectives"][0] == full["objectives"][j]
        assert one["iters"][0] == full["iters"][j]


def test_invalid_inputs_rejected(gmco_mod, small, prob_fp32):
    p, W = small
    bad = W.copy()
    bad[1, 2] = np.nan
    with pytest.raises(gmco_mod.GmcoError) as e:
        prob_fp32.solve_batch(bad, max_iters=5)
    assert e.value.status == 1
    with pytest.raises(gmco_mod.GmcoError):
        prob_fp32.solve_batch(W, t0=-np.ones((8, p.n_dwell), np.float32), max_iters=5)
    with pytest.raises(gmco_mod.GmcoError):
        gmco_mod.Problem(p.A, np.full(p.n_pnt, 7, np.int32), p.params)
    A = p.A.copy()
    A[3, 3] = np.inf
    with pytest.raises(gmco_mod.GmcoError):
        gmco_mod.Problem(A, p.sid, p.params)


def test_device_tensors_and_launch_count(gmco_mod, small, prob_fp32):
    import torch
    p, W = small
    Wd = torch.from_numpy(W).cuda()
    out = prob_fp32.solve_batch(Wd, max_iters=20, tol=0.0)
    assert out["T"].is_cuda and out["objectives"].is_cuda
    host = prob_fp32.solve_batch(W, max_iters=20, tol=0.0)
    assert np.array_equal(out["T"].cpu().numpy(), host["T"])
    assert prob_fp32.last_launch_count() > 20
