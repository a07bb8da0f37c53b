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


def _limit_case(rng, n_pnt, n_dwell, n_struct):
    """Seeded dense case at a size limit: inverse-square-like dose rates (0.002-0.2 Gy/s), so
    that a uniform start gives about 10-40 Gy, structures of uneven size, and per structure a
    lower bound, an upper bound or both around those doses."""
    r2 = rng.uniform(0.5, 12.0, (n_pnt, n_dwell))
    A = (0.1 / r2).astype(np.float32)
    sid = rng.choice(n_struct, n_pnt, p=np.arange(1, n_struct + 1) / (n_struct * (n_struct + 1) / 2))
    sid[:n_struct] = np.arange(n_struct)   # every structure has points
    d_mid = A.sum(axis=1).mean()
    params = np.empty((n_struct, 4))
    for s in range(n_struct):
        kind = s % 3
        lo = d_mid * rng.uniform(0.8, 0.95 if kind == 2 else 1.1) if kind != 1 else -np.inf
        hi = d_mid * rng.uniform(1.05, 1.3) if kind != 0 else np.inf
        params[s] = (rng.uniform(0.5, 2.0), lo, hi, rng.uniform(0.5, 2.0))
    return A, sid.astype(np.int32), params


def _penalty_at(params, sid, w, d):
    """Eq. (1) in FP64 at given doses d: F and h = dF/dd per point."""
    N = np.bincount(sid, minlength=params.shape[0]).astype(np.float64)
    k = (np.asarray(w, np.float64) / N)[sid]
    a, lo, hi, b = (params[sid, c] for c in range(4))
    u = np.maximum(lo - d, 0.0)
    o = np.maximum(d - hi, 0.0)
    return float(np.sum(k * (a * u * u + b * o * o))), 2.0 * k * (b * o - a * u)


# split depth of each form: relative error of A / s and of one dF/dd value in its BF16 terms
SPLIT_EPS = {"bf16x3": 2.0 ** -23, "bf16x2": 2.0 ** -16, "bf16": 2.0 ** -9, "fp8": 2.0 ** -4, "fp32": 0.0}


@pytest.mark.parametrize("form,n_dwell,n_struct", [
    ("bf16x3", 512, 8),   # tensor-core limits: 512 dwells (8 K blocks of 64), 8 structures
    ("bf16x2", 512, 8),
    ("bf16", 512, 8),     # one term of A: 2^-9 relative per element
    ("fp8", 512, 8),      # E4M3 grid of A: 2^-4
    ("fp32", 1024, 16),   # FP32 SIMT limits: the step kernel's widest form
])
def test_size_limits(gmco_mod, oracle_mod, form, n_dwell, n_struct):
    """At the largest sizes each form accepts:

    - doses match the oracle within the form's bound;
    - F is the Eq. (1) sum over the kernel's own doses up to FP32 rounding (1e-6), and the
      gradient is 2 x A^T dF/dd of those doses within the bound its arithmetic gives: the BF16
      split of A and of dF/dd (SPLIT_EPS each) and FP32 accumulation over the points;
    - a short solve reports the oracle's objective at its returned dwell times (zero where it
      meets every bound), below the uniform start's;
    - one dwell or one structure more is refused before any device work."""
    rng = np.random.default_rng(n_dwell + n_struct)
    A, sid, params = _limit_case(rng, 1500, n_dwell, n_struct)
    W = rng.uniform(0.1, 10.0, (6, n_struct)).astype(np.float32)
    X = rng.uniform(0.5, 1.5, (6, n_dwell)).astype(np.float32)
    with gmco_mod.Problem(A, sid, params, precision=form) as pr:
        out = pr.evaluate(W, X, objectives=True, grad=True, dose=True)
        sol = pr.solve_batch(W, max_iters=30, tol=0.0)
    bd = FORMS[form][0] if form in FORMS else 1e-5
    A64 = A.astype(np.float64)
    acc = A.shape[0] * 2.0 ** -24
    for j in range(W.shape[0]):
        _, _, d, _ = oracle_mod.objective(A, sid, params, W[j], X[j])
        dg = out["dose"][j].astype(np.float64)
        assert np.max(np.abs(dg - d) / d) <= bd
        Fg, hg = _penalty_at(params, sid, W[j], dg)
        assert abs(out["objectives"][j] / Fg - 1.0) <= 1e-6, (j, out["objectives"][j], Fg)
        x = X[j].astype(np.float64)
        g_own = 2.0 * x * (A64.T @ hg)
        bound = 2.0 * x * (A64.T @ np.abs(hg)) * (2.0 * SPLIT_EPS[form] + acc)
        err = np.abs(out["grad"][j] - g_own)
        assert np.all(err <= 2.0 * bound + 1e-12 * np.max(np.abs(g_own))), (j, np.max(err / bound))
    for j in range(W.shape[0]):
        F = oracle_mod.objective(A, sid, params, W[j], np.sqrt(sol["T"][j]))[0]
        F0 = oracle_mod.objective(A, sid, params, W[j], np.ones(n_dwell))[0]
        # where the FP32 doses meet every bound (F = 0), the FP64 doses of the same dwell times
        # may cross one by the dose tolerance 1e-5 d: F <= k (1e-5 d)^2, about 1e-8 of the
        # start's k (0.1 d)^2
        tol_f = max(1e-4, FORMS[form][1]) if form in FORMS else 1e-4   # the form's dose error
        assert abs(sol["objectives"][j] - F) <= tol_f * F + 1e-8 * F0
        assert F < F0
    refused = gmco_mod.EUNSUPPORTED if form != "fp32" else gmco_mod.EINVAL
    A2, sid2, params2 = _limit_case(rng, 64, n_dwell + 1, n_struct)
    with pytest.raises(gmco_mod.GmcoError) as e:
        gmco_mod.Problem(A2, sid2, params2, precision=form)
    assert e.value.status == refused
    A3, sid3, params3 = _limit_case(rng, 64, 16, n_struct + 1)
    with pytest.raises(gmco_mod.GmcoError) as e:
        gmco_mod.Problem(A3, sid3, params3, precision=form)
    assert e.value.status == refused


@pytest.mark.parametrize("form", ["fp32", "bf16x3", "bf16x2"])
def test_class_solution_objective(gmco_mod, oracle_mod, form):
    """The paper's full class solution (Table 1: surface and volume point groups of four organs,
    two-sided penalties on every group, eight groups) evaluated and solved: doses, F and the
    gradient against the oracle within the form's bounds, and each solve's reported objective
    equal to the oracle's at its dwell times."""
    from synth import make_class_solution_patient, group_weights
    p = make_class_solution_patient(5)
    rng = np.random.default_rng(5)
    W = group_weights(rng.dirichlet(np.ones(4), 16), p.sid, p.organ)
    X = rng.uniform(0.5, 1.5, (16, p.n_dwell)).astype(np.float32)
    with gmco_mod.Problem(p.A, p.sid, p.params, precision=form) as pr:
        out = pr.evaluate(W, X, objectives=True, grad=True, dose=True)
        sol = pr.solve_batch(W, max_iters=200, tol=1e-9)
    bd, bF, bg = FORMS.get(form, (1e-5, 2e-5, 2e-5))
    ed, eF, eg = _errors(oracle_mod, p.A, p.sid, p.params, W, X, out)
    print(f"class solution {form}: dose {ed:.2e} F {eF:.2e} grad {eg:.2e}")
    assert ed <= bd and eF <= bF and eg <= bg, (ed, eF, eg)
    for j in range(W.shape[0]):
        F = oracle_mod.objective(p.A, p.sid, p.params, W[j], np.sqrt(sol["T"][j]))[0]
        assert abs(sol["objectives"][j] / F - 1.0) <= max(1e-4, bF)
