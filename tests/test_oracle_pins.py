"""Pins of the FP64 oracle against things other than itself (no GPU needed).

Each test fixes a part of the oracle by a hand-computed value, a closed form, an invariant,
a library routine solving a special case, or brute force, so that a plausible slip (a lost
factor, a wrong sign, a transposed operand, an off-by-one in the ring buffer) fails one.
"""
import numpy as np
import pytest
from scipy.optimize import nnls

from synth import make_patient, workload
from tests.conftest import read_fstar

INF = np.inf


# ---------------------------------------------------------------- Eq. (dose), Eq. (1), Eq. (obj)
def test_hand_example_objective_and_gradient(oracle_mod):
    """Four points (one per structure), two dwells, worked by hand.

    x = (2, 1) -> t = (4, 1); A = [[1, 2], [.5, .5], [1, 0], [0, 1]] -> d = (6, 2.5, 4, 1)
    prostate D_min 10: f = (10-6)^2 = 16, f' = -8;   urethra D_max 2: f = .25, f' = 1
    rectum D_max 5: 0;   bladder D_max .5: f = .25, f' = 1
    w = (1, 2, 3, 4), N_s = 1: F = 16 + 2*.25 + 0 + 4*.25 = 17.5
    A^T (w f') = A^T (-8, 2, 0, 4) = (-7, -11);  dF/dx = 2 x (-7, -11) = (-28, -22)
    """
    A = np.array([[1, 2], [0.5, 0.5], [1, 0], [0, 1]], dtype=np.float64)
    sid = np.array([0, 1, 2, 3])
    prm = np.array([[1, 10, INF, 1], [1, -INF, 2, 1], [1, -INF, 5, 1], [1, -INF, 0.5, 1]])
    F, g, d, fs = oracle_mod.objective(A, sid, prm, [1, 2, 3, 4], [2.0, 1.0])
    assert np.array_equal(d, [6, 2.5, 4, 1])
    assert F == 17.5
    assert np.array_equal(g, [-28.0, -22.0])
    assert np.array_equal(fs, [16, 0.25, 0, 0.25])


def test_two_sided_penalty_and_weights(oracle_mod):
    """Eq. (1) with both sides and unequal w_min / w_max (Table 1 style)."""
    prm = np.array([200.0, 15.0, 22.5, 80.0])
    assert oracle_mod.point_penalty(14.0, prm) == 200.0
    assert oracle_mod.point_penalty(15.0, prm) == 0.0
    assert oracle_mod.point_penalty(22.5, prm) == 0.0
    assert oracle_mod.point_penalty(23.5, prm) == 80.0
    assert oracle_mod.point_dpenalty(14.0, prm) == -400.0
    assert oracle_mod.point_dpenalty(23.5, prm) == 160.0
    assert oracle_mod.point_dpenalty(18.0, prm) == 0.0


def test_mean_over_structure_points(oracle_mod):
    """Eq. (obj) divides each structure's sum by its own point count."""
    A = np.array([[1.0], [1.0], [1.0]])
    sid = np.array([0, 0, 1])
    prm = np.array([[1, 3, INF, 1], [1, -INF, 0, 1]])
    # x = 1 -> d = 1 everywhere; structure 0: two points with f = 4 -> mean 4; structure 1: f = 1
    F, _, _, fs = oracle_mod.objective(A, sid, prm, [1.0, 10.0], [1.0])
    assert np.array_equal(fs, [4.0, 1.0]) and F == 14.0


def test_single_source_dose(oracle_mod):
    """d = A t for one dwell: 2 s at 1 cm gives 2 * 0.125754747 Gy (point-source model)."""
    from synth import dose_rate_matrix
    A = dose_rate_matrix(np.array([[0, 0, 1.0], [0.05, 0, 0]]), np.zeros((1, 3)))
    d = oracle_mod.dose(A, [2.0])
    assert d[0] == pytest.approx(2 * 0.125754747, rel=1e-8)
    assert d[1] == pytest.approx(2 * 12.5438793, rel=1e-8)


def test_dose_rate_matrix_pins(oracle_mod):
    """Dose rate matrix of the point-source model: 0.125754747 Gy/s at 1 cm and 12.5438793
    Gy/s at the 0.1 cm clamp (the values above), the same rate anywhere inside the clamp,
    invariance under a common shift and an axis permutation of points and dwells, agreement
    with the input generator's separate numpy evaluation, and refusal where g(r) <= 0."""
    a = oracle_mod.dose_rate([[0, 0, 1.0], [0.05, 0, 0], [0, 0.1, 0], [0, 0, 0]], np.zeros((1, 3)))
    assert a[0, 0] == pytest.approx(0.125754747, rel=1e-8)
    assert a[1, 0] == pytest.approx(12.5438793, rel=1e-8)
    assert a[1, 0] == a[2, 0] == a[3, 0]
    p = make_patient(11, 12, 0.5, (120, 20, 30, 30))
    A = oracle_mod.dose_rate(p.points, p.dwells)
    shift = np.array([3.0, -1.5, 0.25])
    assert np.allclose(oracle_mod.dose_rate(p.points + shift, p.dwells + shift), A, rtol=1e-12, atol=0)
    perm = [2, 0, 1]
    assert np.allclose(oracle_mod.dose_rate(p.points[:, perm], p.dwells[:, perm]), A, rtol=1e-14, atol=0)
    from synth import dose_rate_matrix
    assert np.allclose(A, dose_rate_matrix(p.points, p.dwells), rtol=1e-14, atol=0)
    with pytest.raises(ValueError):
        oracle_mod.dose_rate([[30.0, 0, 0]], np.zeros((1, 3)))


def test_dose_is_exact_matvec(oracle_mod):
    rng = np.random.default_rng(0)
    A = rng.integers(0, 8, size=(37, 11)).astype(np.float64)   # small integers: sums are exact
    t = rng.integers(0, 5, size=11).astype(np.float64)
    assert np.array_equal(oracle_mod.dose(A, t), A @ t)


def test_zero_objective_when_constraints_met(oracle_mod):
    p = make_patient(11, 12, 0.5, (120, 20, 30, 30))
    d0 = p.A.astype(np.float64) @ np.ones(p.n_dwell)
    prm = p.params.copy()
    prm[0, 1] = d0[p.sid == 0].min() - 0.1
    for s in (1, 2, 3):
        prm[s, 2] = d0[p.sid == s].max() + 0.1
    F, g, _, _ = oracle_mod.objective(p.A, p.sid, prm, [1, 2, 3, 4], np.ones(p.n_dwell))
    assert F == 0.0 and np.all(g == 0.0)
    r = oracle_mod.lbfgs(p.A, p.sid, prm, [1, 2, 3, 4], None, max_iters=50, tol=1e-6)
    assert r["status"] == oracle_mod.CONVERGED and r["iters"] == 0 and r["F"] == 0.0
    assert np.array_equal(r["t"], np.ones(p.n_dwell))


def test_gradient_central_differences(oracle_mod):
    p = make_patient(12, 12, 0.5, (300, 50, 80, 80))
    rng = np.random.default_rng(1)
    w = np.array([2.0, 0.7, 1.3, 0.4])
    x = rng.uniform(0.6, 1.6, p.n_dwell)
    F, g, d, _ = oracle_mod.objective(p.A, p.sid, p.params, w, x)
    bounds = np.where(p.sid == 0, p.params[0, 1], p.params[p.sid, 2])
    assert np.min(np.abs(d - bounds)) > 1e-3     # away from the kinks of Eq. (1)
    fd = np.empty_like(x)
    for l in range(p.n_dwell):
        h = 1e-6 * max(1.0, abs(x[l]))
        xp = x.copy(); xp[l] += h
        xm = x.copy(); xm[l] -= h
        fd[l] = (oracle_mod.objective(p.A, p.sid, p.params, w, xp, False)[0]
                 - oracle_mod.objective(p.A, p.sid, p.params, w, xm, False)[0]) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-6 * np.max(np.abs(g))
    # the factor 4 of Eq. (2) (2 from the square, 2 from t = x^2) is what the check pins:
    assert np.max(np.abs(fd - 0.5 * g)) > 0.1 * np.max(np.abs(g))


# ---------------------------------------------------------------- two-loop recursion
def _dense_bfgs_direction(S, Y, order, g):
    """p = -H g with H built by the BFGS inverse update from H0 = gamma I (dense matrices)."""
    n = g.size
    s_new, y_new = S[order[-1]], Y[order[-1]]
    H = (s_new @ y_new) / (y_new @ y_new) * np.eye(n)
    for i in order:   # oldest to newest
        s, y = S[i], Y[i]
        rho = 1.0 / (s @ y)
        V = np.eye(n) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    return -H @ g


@pytest.mark.parametrize("m,count,newest", [(5, 5, 4), (7, 5, 2), (4, 1, 0), (10, 10, 3)])
def test_two_loop_equals_dense_bfgs(oracle_mod, m, count, newest):
    rng = np.random.default_rng(m * 100 + count)
    n = 9
    Q = rng.normal(size=(n, n))
    Htrue = Q @ Q.T + n * np.eye(n)
    S = rng.normal(size=(m, n))
    Y = S @ Htrue.T
    rho = 1.0 / np.einsum("ij,ij->i", S, Y)
    g = rng.normal(size=n)
    order = [(newest - k) % m for k in range(count)][::-1]   # oldest .. newest
    p = oracle_mod.two_loop(S, Y, rho, count, newest, g)
    p_dense = _dense_bfgs_direction(S, Y, order, g)
    assert np.allclose(p, p_dense, rtol=1e-10, atol=1e-12 * np.abs(p_dense).max())
    # secant condition of the newest pair: H y_new = s_new
    if count:
        q = oracle_mod.two_loop(S, Y, rho, count, newest, -Y[newest])
        assert np.allclose(q, S[newest], rtol=1e-9, atol=1e-12)


def test_two_loop_empty_history_is_steepest_descent(oracle_mod):
    g = np.array([1.0, -2.0, 3.0])
    p = oracle_mod.two_loop(np.zeros((3, 3)), np.zeros((3, 3)), np.zeros(3), 0, 2, g)
    assert np.array_equal(p, -g)


# ---------------------------------------------------------------- whole method
def test_convex_quadratic_toy_known_minimiser(oracle_mod):
    """A = diag(a), one two-sided band D_min = D_max = c: t* = c / a, F* = 0."""
    a = np.array([0.5, 1.0, 2.0, 4.0, 0.25])
    A = np.diag(a)
    prm = np.array([[1.0, 3.0, 3.0, 1.0]])
    r = oracle_mod.lbfgs(A, np.zeros(5, np.int32), prm, [1.0], None, max_iters=2000, tol=0.0)
    assert r["F"] < 1e-20
    assert np.allclose(r["t"], 3.0 / a, rtol=1e-9)


def test_nnls_special_case(oracle_mod):
    """Bands with D_min = D_max per structure make Eq. (obj) a weighted NNLS problem:
    min sum_s 1/N_s ||A_s t - c_s||^2 over t >= 0, solved exactly by Lawson-Hanson."""
    rng = np.random.default_rng(3)
    A = rng.uniform(0.0, 1.0, size=(40, 6)) ** 3
    A[20:, 0] += 2.0                        # dwell 0 mostly irradiates the low-target structure
    sid = np.array([0] * 20 + [1] * 20)
    prm = np.array([[1.0, 3.0, 3.0, 1.0], [1.0, 0.5, 0.5, 1.0]])
    b = np.where(sid == 0, 3.0, 0.5)
    scale = np.sqrt(1.0 / 20.0)
    t_ref, res = nnls(scale * A, scale * b)
    F_ref = res ** 2
    assert np.sum(t_ref == 0) >= 1    # the bound is active, so non-negativity matters
    r = oracle_mod.lbfgs(A, sid, prm, [1.0, 1.0], None, max_iters=20000, tol=1e-15)
    assert r["F"] == pytest.approx(F_ref, rel=1e-7)
    assert np.allclose(r["t"], t_ref, atol=1e-3)


def _grid_min(oracle_mod, A, sid, prm, w, tmax, n=21, zooms=12):
    lo = np.zeros(A.shape[1])
    hi = np.full(A.shape[1], tmax)
    best = (np.inf, None)
    for _ in range(zooms):
        axes = [np.linspace(lo[k], hi[k], n) for k in range(A.shape[1])]
        grid = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, A.shape[1])
        for t in grid:
            F = oracle_mod.objective(A, sid, prm, w, np.sqrt(t), False)[0]
            if F < best[0]:
                best = (F, t)
        step = (hi - lo) / (n - 1)
        lo = np.maximum(best[1] - 3 * step, 0.0)
        hi = best[1] + 3 * step
    return best


def test_brute_force_three_dwells(oracle_mod):
    p = make_patient(21, 12, 0.5, (120, 20, 30, 30))
    cols = [10, 40, 77]
    A = p.A[:, cols].astype(np.float64) * 4.0
    w = np.array([3.0, 1.0, 0.5, 0.5])
    Fg, tg = _grid_min(oracle_mod, A, p.sid, p.params, w, tmax=400.0, n=17, zooms=16)
    r = oracle_mod.lbfgs(A, p.sid, p.params, w, None, max_iters=5000, tol=1e-15)
    assert r["F"] <= Fg * (1 + 1e-9)
    assert r["F"] >= Fg * (1 - 1e-6)


def test_kkt_and_exact_optimum(oracle_mod):
    """The oracle's long run and the exact active-set optimum agree and satisfy KKT."""
    p, W, _ = workload("prostate-2k-8plans")
    fstar = read_fstar("prostate-2k-8plans")
    j = 0
    r = oracle_mod.lbfgs(p.A, p.sid, p.params, W[j], None, max_iters=20000, tol=1e-15)
    assert r["F"] == pytest.approx(fstar[j], rel=1e-6)
    assert oracle_mod.kkt_residual(p.A, p.sid, p.params, W[j], r["t"]) < 1e-4
    ex = oracle_mod.fstar(p.A, p.sid, p.params, W[j])
    assert ex["kkt"] < 1e-10
    assert ex["F"] == pytest.approx(fstar[j], rel=1e-12)


def test_random_start_invariance(oracle_mod):
    """Random starts in [0, 10] s reach the same optimum (convexity; Sec. 3.1.1 reports
    agreement within 0.02 % from 1000 random starts)."""
    p, W, _ = workload("prostate-2k-8plans")
    fstar = read_fstar("prostate-2k-8plans")
    j = 5
    rng = np.random.default_rng(5)
    T0 = rng.uniform(0.0, 10.0, size=(8, p.n_dwell))
    Wj = np.tile(W[j], (8, 1))
    r = oracle_mod.lbfgs_batch(p.A, p.sid, p.params, Wj, T0, max_iters=20000, tol=1e-15)
    assert fstar[j] > 0
    assert np.all(np.abs(r["F"] / fstar[j] - 1.0) < 2e-4)


def test_armijo_and_monotone_trace(oracle_mod):
    p, W, _ = workload("prostate-2k-8plans")
    r = oracle_mod.lbfgs(p.A, p.sid, p.params, W[3], None, max_iters=300, tol=0.0, trace=True)
    tr = r["trace"]
    F, alpha, gtp = tr[:, 0], tr[:, 1], tr[:, 2]
    assert np.all(np.diff(F) < 0)
    assert np.all(F[1:] <= F[:-1] + 1e-4 * alpha[1:] * gtp[1:])
    assert np.all(gtp[1:] < 0)


def test_weight_scaling_is_exact(oracle_mod):
    """F(4 w) = 4 F(w) along an identical trajectory (powers of two scale exactly)."""
    p, W, _ = workload("prostate-2k-8plans")
    w = W[1].astype(np.float64)
    r1 = oracle_mod.lbfgs(p.A, p.sid, p.params, w, None, max_iters=60, tol=0.0)
    r4 = oracle_mod.lbfgs(p.A, p.sid, p.params, 4.0 * w, None, max_iters=60, tol=0.0)
    g0 = oracle_mod.objective(p.A, p.sid, p.params, w, np.ones(p.n_dwell))[1]
    assert np.abs(g0).max() >= 1.0          # first step alpha0 = 1/|g|inf in both runs
    assert r4["F"] == 4.0 * r1["F"]
    assert np.array_equal(r4["t"], r1["t"])


def test_dwell_permutation_equivariance(oracle_mod):
    p, W, _ = workload("prostate-2k-8plans")
    perm = np.random.default_rng(2).permutation(p.n_dwell)
    r = oracle_mod.lbfgs(p.A, p.sid, p.params, W[0], None, max_iters=10, tol=0.0)
    rp = oracle_mod.lbfgs(p.A[:, perm], p.sid, p.params, W[0], None, max_iters=10, tol=0.0)
    assert rp["F"] == pytest.approx(r["F"], rel=1e-10)
    assert np.allclose(rp["t"], r["t"][perm], rtol=1e-8)


def test_max_iters_zero_and_status(oracle_mod):
    p, W, _ = workload("prostate-2k-8plans")
    r = oracle_mod.lbfgs(p.A, p.sid, p.params, W[0], None, max_iters=0, tol=1e-6)
    assert r["status"] == oracle_mod.MAXITER and r["iters"] == 0
    assert np.array_equal(r["t"], np.ones(p.n_dwell))
    nan_w = W[0].astype(np.float64).copy()
    nan_w[2] = np.nan
    r = oracle_mod.lbfgs(p.A, p.sid, p.params, nan_w, None, max_iters=5, tol=1e-6)
    assert r["status"] == oracle_mod.NONFINITE



def test_evaluation_budget_stops_on_the_same_path(oracle_mod):
    """max_evals bounds the objective evaluations (the first one and every line-search trial):
    the capped run takes exactly the uncapped run's path and stops at its last accepted point
    once the next trial would exceed the budget."""
    p, W, _ = workload("prostate-2k-8plans")
    runs = [oracle_mod.lbfgs(p.A, p.sid, p.params, W[j], None, max_iters=150, tol=0.0, trace=True)
            for j in range(8)]
    j = int(np.argmax([r["evals"] - r["iters"] for r in runs]))
    full = runs[j]
    assert full["evals"] > full["iters"] + 1          # this path has rejected trials
    for cap in (1, 2, 9, 40, full["evals"] - 1, full["evals"]):
        r = oracle_mod.lbfgs(p.A, p.sid, p.params, W[j], None, max_iters=150, tol=0.0, max_evals=cap)
        assert r["evals"] == cap and r["status"] == oracle_mod.MAXITER
        assert r["F"] == full["trace"][r["iters"], 0]
        assert r["iters"] <= cap - 1
    r = oracle_mod.lbfgs(p.A, p.sid, p.params, W[j], None, max_iters=150, tol=0.0, max_evals=0)
    assert r["evals"] == full["evals"] and r["F"] == full["F"]

def test_stop_window_is_the_first_run_of_small_changes(oracle_mod):
    """Sec. 2.2.3's stop rule over a window of w accepted iterations: the run stops at the first
    iteration k whose last w relative objective changes |F_(i-1) - F_i| / |F_(i-1)| are all
    <= tol, along the path that a run without the stop rule takes (the window changes when
    the path ends, not the path)."""
    p, W, _ = workload("prostate-2k-8plans")
    tol = 1e-3
    for j in (0, 3, 6):
        full = oracle_mod.lbfgs(p.A, p.sid, p.params, W[j], None, max_iters=400, tol=0.0,
                                trace=True)
        F = full["trace"][:, 0]
        small = np.abs(F[:-1] - F[1:]) <= tol * np.abs(F[:-1])   # small[i]: iteration i + 1
        for w in (1, 2, 3, 5):
            r = oracle_mod.lbfgs(p.A, p.sid, p.params, W[j], None, max_iters=400, tol=tol,
                                 stop_window=w)
            run, expect = 0, None
            for i, ok in enumerate(small):
                run = run + 1 if ok else 0
                if run >= w:
                    expect = i + 1
                    break
            assert expect is not None and expect < 400
            assert r["status"] == oracle_mod.CONVERGED and r["iters"] == expect, (j, w, r["iters"], expect)
            assert r["F"] == F[expect]


# ---------------------------------------------------------------- DVH indices
def test_dvh_hand_made(oracle_mod):
    pro = np.arange(2.0, 21.0, 2.0)            # 2, 4, ..., 20 (N = 10)
    ure = np.arange(10.0, 20.0)                # 10 .. 19
    rec = np.array([11.25, 11.24, 12.0])
    bla = np.array([0.0])
    d = np.concatenate([pro, ure, rec, bla])
    sid = np.array([0] * 10 + [1] * 10 + [2] * 3 + [3])
    out = oracle_mod.dvh(d, sid, 4, 15.0)
    assert out[0] == 30.0                       # 16, 18, 20 >= 15 Gy
    assert out[1] == pytest.approx(100 * 4.0 / 15.0)   # k = ceil(9) = 9th largest = 4 Gy
    assert out[2] == pytest.approx(100 * 19.0 / 15.0)  # k = ceil(1) = 1: the maximum
    assert out[3] == pytest.approx(200.0 / 3.0)        # 11.25 and 12 >= 11.25
    assert out[4] == 0.0
    # k = ceil(0.9 N) with N = 7: k = 7 (6.3 rounds up), the minimum
    d7 = np.array([5.0, 1.0, 7.0, 3.0, 2.0, 6.0, 4.0])
    assert oracle_mod.dvh(d7, np.zeros(7, np.int32), 1, 10.0)[1] == pytest.approx(10.0)
    assert np.isnan(oracle_mod.dvh(d7, np.zeros(7, np.int32), 1, 10.0)[2])


def test_rtog_classes_and_selection_hand_made(oracle_mod):
    """Plan evaluation at each criterion's boundary (V100 >= 90 % and >= 95 % for RTOG+,
    urethra D10 < 118 %, rectum and bladder V75 < 1 cc) and the selection order: RTOG+ valid,
    then RTOG valid, each by the highest V100; with none valid, the lowest rectum + bladder V75
    among plans meeting the target and urethra criteria (else among all), first index on ties.
    Volumes 50 cc (rectum) and 100 cc (bladder): 1 cc is 2 % and 1 %."""
    ok = [0.5, 0.5]
    rows = [[90.0, 100, 117.9] + ok,      # RTOG: V100 exactly at 90 %
            [95.0, 100, 117.9] + ok,      # RTOG+: exactly at 95 %
            [89.99, 100, 110] + ok,       # target fails
            [99.0, 100, 118.0] + ok,      # urethra D10 exactly 118 % fails
            [99.0, 100, 110, 2.0, 0.5],   # rectum exactly 1 cc fails
            [99.0, 100, 110, 0.5, 1.0],   # bladder exactly 1 cc fails
            [99.0, 100, 110, 1.99, 0.99]]  # both just below 1 cc: RTOG+
    cls, sel = oracle_mod.rtog_select(rows, 50.0, 100.0)
    assert list(cls) == [1, 2, 0, 0, 0, 0, 2]
    assert sel == 6                                   # RTOG+ with the higher V100 (99 > 95)
    cls, sel = oracle_mod.rtog_select([rows[0], [93.0, 100, 100] + ok, [93.0, 100, 100] + ok], 50.0, 100.0)
    assert list(cls) == [1, 1, 1] and sel == 1        # highest V100, first of equals
    invalid = [[99.0, 100, 120, 0.2, 0.2],            # urethra fails: set aside while others pass
               [91.0, 100, 110, 4.0, 3.0],            # 2 + 3 cc
               [92.0, 100, 110, 3.0, 2.0],            # 1.5 + 2 cc: the lowest
               [80.0, 100, 110, 0.0, 0.0]]            # target fails
    cls, sel = oracle_mod.rtog_select(invalid, 50.0, 100.0)
    assert list(cls) == [0, 0, 0, 0] and sel == 2
    cls, sel = oracle_mod.rtog_select([invalid[0], invalid[3]], 50.0, 100.0)
    assert sel == 1                                   # none meets target and urethra: lowest V75


def test_pareto_front_hand_made(oracle_mod):
    """(1,3), (2,2), (3,1) are non-dominated, (2,3) is dominated by (2,2) and (1,3), (4,4) by
    all; equal rows do not dominate each other; with one objective only the minima remain."""
    obj = [[1, 3], [2, 2], [3, 1], [2, 3], [4, 4], [2, 2]]
    assert list(oracle_mod.pareto(obj)) == [1, 1, 1, 0, 0, 1]
    assert list(oracle_mod.pareto([[3.0], [1.0], [2.0], [1.0]])) == [0, 1, 0, 1]
    rng = np.random.default_rng(0)
    o = rng.integers(0, 6, size=(60, 3)).astype(float)
    nd = oracle_mod.pareto(o).astype(bool)
    # every plan off the front is dominated by a plan on it (dominance is transitive)
    for i in np.where(~nd)[0]:
        assert any(np.all(o[j] <= o[i]) and np.any(o[j] < o[i]) for j in np.where(nd)[0])
