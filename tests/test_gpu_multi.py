"""Several patients of uneven size solved with one launch per GEMM and per update per step
(gmco_solve_multi), against per-patient solves and the FP64 oracle."""
import numpy as np
import pytest

from synth import make_patient, weights_dirichlet, weights_loguniform

pytestmark = pytest.mark.gpu

# (seed, catheters, dwell step, points per structure, scale) and plans per patient:
# 96 / 224 / 352 / 72 dwells (352: three dwell tiles of the gradient GEMM),
# 5 to 130 plans (130: two plan tiles of the dose GEMM, and of the gradient GEMM with
# 128-plan tiles), 760 to 4000 points.
SPECS = [
    ((11, 12, 0.5, (900, 150, 250, 250), 1.0), 5),
    ((12, 14, 0.25, (2500, 300, 600, 600), 1.1), 130),
    ((13, 16, 0.2, (1800, 250, 500, 450), 1.2), 37),
    ((14, 9, 0.4, (480, 60, 110, 110), 0.8), 8),
]


@pytest.fixture(scope="module")
def patients():
    out = []
    for (seed, ncat, step, npts, scale), P in SPECS:
        p = make_patient(seed, ncat, step, npts, scale)
        W = weights_loguniform(seed, P)
        out.append((p, W))
    assert sorted(p.n_dwell for p, _ in out) == [72, 96, 224, 352]
    return out


def _problems(gmco_mod, patients, precision="bf16x2", **opt):
    return [gmco_mod.Problem(p.A, p.sid, p.params, precision=precision, **opt)
            for p, _ in patients]


@pytest.mark.parametrize("split,tile", [(3, 0), (0, 0), (3, 128)])
def test_multi_equals_per_patient_bitwise(gmco_mod, patients, split, tile):
    """Every patient's T, objectives, iterations and status equal those of its own
    gmco_solve_batch with the same split length and gradient tile, bit for bit."""
    # the multi launch forms every gradient with the GEMM: so do the per-patient solves here
    probs = _problems(gmco_mod, patients, grad_split_kb=split, grad_plan_tile=tile,
                      sparse_grad_permille=0)
    Ws = [W for _, W in patients]
    with gmco_mod.Multi(probs) as mu:
        assert mu.tiles == (16, tile)          # the problems' tile option is the initial value
        mu.tiles = (split, tile)
        res = mu.solve(Ws, max_iters=40, tol=1e-7)
        launches = mu.last_launch_count()
    for (p, W), pr, r in zip(patients, probs, res):
        ref = pr.solve_batch(W, max_iters=40, tol=1e-7)
        for k in ("T", "objectives", "iters", "status", "dvh"):
            assert np.array_equal(r[k], ref[k], equal_nan=True), (p.n_dwell, k)
    # per step: one dose GEMM, one gradient GEMM and one update for all patients
    steps = max(int(r["iters"].max()) for r in res)
    assert launches < 3 * 2 * 31 * (steps + 2) + 40 * len(probs)
    for pr in probs:
        pr.close()


def test_multi_results_against_oracle(gmco_mod, oracle_mod, patients):
    """Reported objectives are the FP32 objective of the returned T (checked with the FP64
    oracle), the solve decreases every objective from the uniform start, and the first
    iterations follow the oracle's (FP64) path."""
    probs = _problems(gmco_mod, patients, precision="bf16x3")
    Ws = [W for _, W in patients]
    with gmco_mod.Multi(probs) as mu:
        r5 = mu.solve(Ws, max_iters=3, tol=0.0)
        res = mu.solve(Ws, max_iters=60, tol=1e-7)
    for (p, W), a, b in zip(patients, r5, res):
        for j in range(0, W.shape[0], max(1, W.shape[0] // 6)):
            F5 = oracle_mod.objective(p.A, p.sid, p.params, W[j], np.sqrt(a["T"][j]))[0]
            assert abs(a["objectives"][j] / F5 - 1.0) < 1e-5
            ref = oracle_mod.lbfgs(p.A, p.sid, p.params, W[j], None, max_iters=3, tol=0.0)
            assert abs(a["objectives"][j] / ref["F"] - 1.0) < 1e-3, (p.n_dwell, j)
            F = oracle_mod.objective(p.A, p.sid, p.params, W[j], np.sqrt(b["T"][j]))[0]
            F0 = oracle_mod.objective(p.A, p.sid, p.params, W[j], np.ones(p.n_dwell))[0]
            assert abs(b["objectives"][j] / F - 1.0) < 1e-5
            assert F < F0
    for pr in probs:
        pr.close()


def test_autotune_picks_a_candidate(gmco_mod, patients):
    probs = _problems(gmco_mod, patients)
    Ws = [W for _, W in patients]
    with gmco_mod.Multi(probs) as mu:
        best, ms = mu.autotune(Ws, steps=4, candidates=(0, 2, 8))
        assert best in (0, 2, 8) and mu.split == best
        assert all(np.isfinite(v) and v > 0 for v in ms.values())
        assert ms[best] == min(ms.values())
        # the tuned object solves normally afterwards
        res = mu.solve(Ws, max_iters=5, tol=0.0)
    assert all(np.all(r["iters"] == 5) for r in res)
    for pr in probs:
        pr.close()


def test_autotune_tiles_picks_a_candidate(gmco_mod, patients):
    """The tile autotuner times (split length, gradient plan tile) pairs, keeps the fastest,
    and the tuned launch gives the same results as a launch set to that pair by hand."""
    probs = _problems(gmco_mod, patients)
    Ws = [W for _, W in patients]
    cands = ((0, 0), (8, 128), (8, 256))
    with gmco_mod.Multi(probs) as mu:
        best, ms = mu.autotune_tiles(Ws, steps=4, candidates=cands)
        assert best in cands and mu.tiles == best
        assert ms[best] == min(ms.values()) and all(np.isfinite(v) and v > 0 for v in ms.values())
        tuned = mu.solve(Ws, max_iters=8, tol=0.0)
        mu.tiles = best
        again = mu.solve(Ws, max_iters=8, tol=0.0)
    for a, b in zip(tuned, again):
        for k in ("T", "objectives", "iters"):
            assert np.array_equal(a[k], b[k])
    for pr in probs:
        pr.close()


def test_multi_rejects_bad_groups(gmco_mod, patients):
    p, _ = patients[0]
    a = gmco_mod.Problem(p.A, p.sid, p.params, precision="bf16x2")
    b = gmco_mod.Problem(p.A, p.sid, p.params, precision="bf16")
    c = gmco_mod.Problem(p.A, p.sid, p.params, precision="fp32")
    with pytest.raises(gmco_mod.GmcoError) as e:
        gmco_mod.Multi([a, b])
    assert e.value.status == gmco_mod.EINVAL
    with pytest.raises(gmco_mod.GmcoError) as e:
        gmco_mod.Multi([c])
    assert e.value.status == gmco_mod.EUNSUPPORTED
    with pytest.raises(gmco_mod.GmcoError) as e:
        gmco_mod.Multi([a, a])
    assert e.value.status == gmco_mod.EINVAL
    with gmco_mod.Multi([a]) as mu:
        with pytest.raises(gmco_mod.GmcoError):
            mu.solve([np.full((3, 4), -1.0, np.float32)], max_iters=2)
    for x in (a, b, c):
        x.close()


def test_wide_patient_evaluate(gmco_mod, oracle_mod):
    """460 dwells: two MMA widths in one gradient accumulator that takes both TMEM buffers.
    Doses to 1e-5.  F and the gradient sum squared (or linear) violations, which are small
    differences of large doses, so the dose error of the tensor-core accumulation (about 20
    bits over 460 products; measured 5.7e-6) is amplified there: bound 6e-5 (measured
    2.7e-5).  The FP32 SIMT form, printed beside it, accumulates exactly in FP32 order."""
    p = make_patient(21, 20, 0.2, (1500, 200, 400, 400), 1.3)
    assert p.n_dwell == 460
    rng = np.random.default_rng(21)
    W = weights_dirichlet(21, 40)
    X = rng.uniform(0.3, 1.5, (40, p.n_dwell)).astype(np.float32)
    errs = {}
    for form in ("bf16x3", "fp32"):
        with gmco_mod.Problem(p.A, p.sid, p.params, precision=form) as pr:
            out = pr.evaluate(W, X, objectives=True, grad=True, dose=True)
        ed = eF = eg = 0.0
        for j in range(0, 40, 7):
            F, g, d, _ = oracle_mod.objective(p.A, p.sid, p.params, W[j], X[j])
            ed = max(ed, np.max(np.abs(out["dose"][j] - d) / d))
            eF = max(eF, abs(out["objectives"][j] / F - 1.0))
            eg = max(eg, np.max(np.abs(out["grad"][j] - g)) / np.max(np.abs(g)))
        errs[form] = (ed, eF, eg)
        print(form, "dose %.2e F %.2e grad %.2e" % errs[form])
    ed, eF, eg = errs["bf16x3"]
    assert ed < 1e-5
    assert eF < 6e-5 and eg < 6e-5
    assert errs["fp32"][0] < 1e-5
