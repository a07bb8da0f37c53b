"""Tensor-core (tcgen05) precision forms vs the FP64 oracle, through the C ABI.

Bounds follow the BF16 split depth: one term keeps 8 significand bits of A / s (relative
error <= 2^-9 per element), two terms about 16, three terms the full FP32 significand; E4M3
keeps 4 bits.  Dose errors are relative per point; F and the gradient relative to their scale.
"""
import numpy as np
import pytest

from synth import make_patient, workload
from tests.conftest import read_fstar

pytestmark = pytest.mark.gpu

FORMS = {  # name: (dose rel, F rel, grad rel to max |g|)
    "bf16": (4e-3, 8e-3, 2e-2),
    "fp8": (7e-2, 1.5e-1, 3e-1),
    "bf16x2": (3e-5, 6e-5, 2e-4),
    "bf16x3": (1e-5, 1e-5, 1e-5),
}


def _errors(oracle_mod, A, sid, prm, W, X, out):
    ed, eF, eg = 0.0, 0.0, 0.0
    for j in range(W.shape[0]):
        F, g, d, _ = oracle_mod.objective(A, sid, prm, W[j], X[j])
        ed = max(ed, np.max(np.abs(out["dose"][j] - d) / np.maximum(np.abs(d), 1e-30)))
        eF = max(eF, abs(out["objectives"][j] - F) / F)
        eg = max(eg, np.max(np.abs(out["grad"][j] - g)) / np.max(np.abs(g)))
    return ed, eF, eg


@pytest.mark.parametrize("form", list(FORMS))
def test_evaluate_error_bounds(gmco_mod, oracle_mod, form):
    p, W, _ = workload("prostate-2k-8plans")
    X = np.random.default_rng(0).uniform(0.5, 1.5, (8, p.n_dwell)).astype(np.float32)
    with gmco_mod.Problem(p.A, p.sid, p.params, precision=form) as pr:
        out = pr.evaluate(W, X, objectives=True, grad=True, dose=True)
    ed, eF, eg = _errors(oracle_mod, p.A, p.sid, p.params, W, X, out)
    print(f"{form}: dose {ed:.2e} F {eF:.2e} grad {eg:.2e}")
    bd, bF, bg = FORMS[form]
    assert ed <= bd and eF <= bF and eg <= bg, (form, ed, eF, eg)


@pytest.mark.parametrize("form", ["bf16", "bf16x3"])
def test_evaluate_ragged(gmco_mod, oracle_mod, form):
    """n_pnt = 1037, n_dwell = 45 (neither a tile multiple), 200 plans (two plan tiles)."""
    p = make_patient(4, 12, 0.5, (700, 100, 150, 150))
    rng = np.random.default_rng(4)
    rows = np.sort(rng.permutation(p.n_pnt)[:1037])
    A = np.ascontiguousarray(p.A[rows][:, :45])
    sid = p.sid[rows]
    W = (10.0 ** rng.uniform(-1, 1, (200, 4))).astype(np.float32)
    X = rng.uniform(0.3, 2.0, (200, 45)).astype(np.float32)
    with gmco_mod.Problem(A, sid, p.params, precision=form) as pr:
        out = pr.evaluate(W, X, objectives=True, grad=True, dose=True)
    ed, eF, eg = _errors(oracle_mod, A, sid, p.params, W, X, out)
    bd, bF, bg = FORMS[form]
    assert ed <= bd and eF <= bF and eg <= bg, (form, ed, eF, eg)


@pytest.mark.parametrize("form", ["bf16x3", "fp32"])
def test_paper_scale_sampled(gmco_mod, oracle_mod, form):
    """12000 points x 324 dwells x 1000 plans (the benchmark's launch shape), sampled plans.

    Dose within 1e-5 per point; F and the gradient within 2e-5: both sum 12000 FP32 terms
    (the SIMT FP32 form is held to the same bound)."""
    p, W, _ = workload("prostate-12k-1000plans")
    X = np.random.default_rng(1).uniform(0.2, 1.5, (1000, p.n_dwell)).astype(np.float32)
    with gmco_mod.Problem(p.A, p.sid, p.params, precision=form) as pr:
        out = pr.evaluate(W, X, objectives=True, grad=True, dose=True)
    idx = [0, 127, 128, 511, 999]
    ed, eF, eg = _errors(oracle_mod, p.A, p.sid, p.params, W[idx], X[idx],
                         {k: v[idx] for k, v in out.items()})
    print(f"paper scale {form}: dose {ed:.2e} F {eF:.2e} grad {eg:.2e}")
    assert ed <= 1e-5 and eF <= 2e-5 and eg <= 2e-5, (ed, eF, eg)


def test_bf16x3_solve_reaches_exact_optimum(gmco_mod, oracle_mod):
    p, W, _ = workload("prostate-2k-8plans")
    fstar = read_fstar("prostate-2k-8plans")
    with gmco_mod.Problem(p.A, p.sid, p.params, precision="bf16x3") as pr:
        out = pr.solve_batch(W, max_iters=20000, tol=1e-10)
    gaps = []
    for j in range(8):
        F = oracle_mod.objective(p.A, p.sid, p.params, W[j], np.sqrt(out["T"][j]))[0]
        assert abs(out["objectives"][j] / F - 1.0) <= 1e-5
        gaps.append(F / fstar[j] - 1.0)
    print("bf16x3 gaps", gaps, out["iters"], out["status"])
    # The tensor cores accumulate in FP32 with truncation, so some plans stop on the relative-
    # change rule a little above 1e-4 (at paper scale about 62 % of plans reach 1e-4 under the
    # same rule, 98 % with the FP32 form); which ones varies with the summation order.
    assert min(gaps) >= -1e-9
    assert sum(g <= 1e-4 for g in gaps) >= 5
    assert max(gaps) <= 2e-3


@pytest.mark.parametrize("form", ["bf16x2", "bf16x3"])
def test_active_set_gradient_solve(gmco_mod, oracle_mod, form):
    """Solves whose gradient is formed from the active (plan, point) pairs alone on every step
    after the first (threshold 1000 per thousand) reach the exact optimum as the gradient
    GEMM's solves do; the objective each reports is the oracle's at its returned dwell times."""
    p, W, _ = workload("prostate-2k-8plans")
    fstar = read_fstar("prostate-2k-8plans")
    res = {}
    for perm in (0, 1000):
        with gmco_mod.Problem(p.A, p.sid, p.params, precision=form,
                              sparse_grad_permille=perm) as pr:
            out = pr.solve_batch(W, max_iters=20000, tol=1e-10)
            res[perm] = (out, pr.last_sparse_steps())
    (out0, s0), (out1, s1) = res[0], res[1000]
    assert s0 == -1
    assert s1 > 0 and s1 >= int(out1["iters"].max()) - 1, (s1, out1["iters"])
    tol_f = FORMS[form][1]
    gaps = {0: [], 1000: []}
    for perm, (out, _) in res.items():
        for j in range(W.shape[0]):
            F = oracle_mod.objective(p.A, p.sid, p.params, W[j], np.sqrt(out["T"][j]))[0]
            assert abs(out["objectives"][j] / F - 1.0) <= tol_f, (perm, j)
            gaps[perm].append(F / fstar[j] - 1.0)
    print(form, "GEMM gaps", gaps[0], "active-set gaps", gaps[1000], out1["iters"], out1["status"])
    assert min(gaps[1000]) >= -1e-9
    assert sum(g <= 1e-4 for g in gaps[1000]) >= sum(g <= 1e-4 for g in gaps[0]) - 1
    assert max(gaps[1000]) <= 2e-3


def test_active_set_gradient_engages_at_three_percent(gmco_mod):
    """With a threshold of 30 per thousand a long solve takes most of its steps on the
    active-set gradient (the active pairs fall to a few per cent of the points), and the
    results are reproducible bit for bit."""
    p, W, _ = workload("prostate-2k-8plans")
    outs = []
    with gmco_mod.Problem(p.A, p.sid, p.params, precision="bf16x2",
                          sparse_grad_permille=30) as pr:
        for _ in range(2):
            out = pr.solve_batch(W, max_iters=300, tol=1e-9)
            outs.append((out, pr.last_sparse_steps()))
    (a, sa), (b, sb) = outs
    assert sa == sb and sa > int(a["iters"].max()) // 2, (sa, a["iters"])
    for k in ("T", "objectives", "iters", "status"):
        assert np.array_equal(a[k], b[k]), k
