"""Solve-level parity of the GPU path against the FP64 oracle, through the C ABI.

(a) The headline form (bf16x2) reaches the exact optimum F* on as many plans as the oracle's
    own L-BFGS does under the same stopping rule, and every reported objective is the plan's
    Eq. (obj) value at the returned dwell times.
(b) The iteration path past the wrap of the m-pair history ring (Sec. 2.2.2; the two-loop
    recursion reads the pairs newest to oldest) follows the oracle's.
(c) DVH indices (Sec. 2.3.1) of converged plans against those of the exact optimum.
(d) The stop rule with a window of several iterations (Sec. 2.2.3's relative variation,
    required on stop_window consecutive accepted iterations).

The L-BFGS trajectory is chaotic: the oracle itself, given a dose-rate matrix perturbed by a
relative 2^-22, ends 25 iterations 1e-2 away in F on the prostate workload.  So (b) and (d)
run on a smooth variant (every structure an equality band D_min = D_max, so no point crosses
a kink of Eq. (1)) and take their tolerance from the oracle's own sensitivity: the GPU must
agree with the oracle within ten times what the oracle agrees with itself under a relative
perturbation of A of 2^-16.  That is the size of the two forms' own errors: their doses are
within 1.5e-6 (FP32) and 2.2e-6 (bf16x3) of the oracle's per point, and their gradients, sums
of terms of both signs, within about 1e-5 of the largest term, i.e. 2^-16.6.
The stored values of (a) and (c) are written by tests/golden/make_converged.py (oracle only).
"""
import math
import os

import numpy as np
import pytest

from synth import workload
from tests.conftest import ROOT, read_fstar

pytestmark = pytest.mark.gpu

QUALITY = 1e-4
RULE = dict(tol=1e-10, max_iters=3000)
MAX_EVALS = 3000
FORM_EPS = {"fp32": 2.0 ** -16, "bf16x3": 2.0 ** -16}
FLOOR_F = {"fp32": 1e-5, "bf16x3": 1e-5}   # the forms' objective error bound (evaluation tests)
FLOOR_T = {"fp32": 1e-5, "bf16x3": 1e-4}
# the reported objective is the FP32 re-evaluation at the returned T: its error against
# Eq. (obj) in FP64 is 1e-5 on the small workload and up to 6e-5 at 12 000 points (the
# evaluation tests' bounds), where objectives near the optimum are small sums of squares
REPORT_TOL = {"prostate-2k-8plans": 1e-5, "prostate-12k-1000plans": 6e-5}


def read_converged(name):
    rows = {}
    with open(os.path.join(ROOT, "tests", "golden", f"converged_{name}.txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            a = line.split()
            rows[int(a[0])] = dict(F=float(a[1]), iters=int(a[2]), status=int(a[3]),
                                   v100=float(a[4]), d90=float(a[5]), Fstar=float(a[6]),
                                   v100_star=float(a[7]), d90_star=float(a[8]))
    return rows


def smooth_params(params):
    """Equality bands (w, c, c, w) per structure: F is a smooth quadratic of the doses."""
    prm = np.array(params, dtype=np.float64)
    for s, c in enumerate((15.0, 13.0, 9.0, 8.0)[: prm.shape[0]]):
        prm[s] = (1.0, c, c, 1.0)
    return prm


def oracle_self_spread(oracle_mod, A, sid, prm, W, eps, **kw):
    """The oracle's runs at A and at A (1 + eps u), u uniform in [-1, 1] (seeded): per plan the
    two results, the relative F difference and the T difference over max |T|."""
    rng = np.random.default_rng(7)
    A2 = np.asarray(A, np.float64) * (1.0 + eps * rng.uniform(-1.0, 1.0, A.shape))
    out = []
    for j in range(W.shape[0]):
        r = oracle_mod.lbfgs(A, sid, prm, W[j], None, **kw)
        r2 = oracle_mod.lbfgs(A2, sid, prm, W[j], None, **kw)
        out.append(dict(r=r, r2=r2, dF=abs(r2["F"] / r["F"] - 1.0),
                        dT=float(np.max(np.abs(r2["t"] - r["t"])) / np.max(np.abs(r["t"])))))
    return out


_SOLVED = {}


def _solve_sample(gmco_mod, name):
    """The bf16x2 solve of the golden sample under the benchmark's rule (once per module)."""
    if name not in _SOLVED:
        p, W, _ = workload(name)
        conv = read_converged(name)
        idx = np.array(sorted(conv))
        with gmco_mod.Problem(p.A, p.sid, p.params, precision="bf16x2",
                              max_evals=MAX_EVALS) as pr:
            out = pr.solve_batch(W[idx], allow_timeout=True, **RULE)
        _SOLVED[name] = (p, W, idx, conv, out)
    return _SOLVED[name]


def _solve_quality(gmco_mod, oracle_mod, name, n_expected):
    p, W, idx, conv, out = _solve_sample(gmco_mod, name)
    assert len(idx) == n_expected
    fstar = read_fstar(name)
    gpu_ok = ora_ok = 0
    gaps = []
    for r, j in enumerate(idx):
        F_o = oracle_mod.objective(p.A, p.sid, p.params, W[j], np.sqrt(out["T"][r]))[0]
        # the reported objective is the FP32 re-evaluation at the returned T: Eq. (obj) there
        assert abs(out["objectives"][r] / F_o - 1.0) <= REPORT_TOL[name], (j, out["objectives"][r], F_o)
        assert abs(conv[j]["Fstar"] / fstar[j] - 1.0) <= 1e-9   # the two golden files agree
        gap = F_o / fstar[j] - 1.0
        assert gap >= -1e-9, (j, gap)                              # nothing beats F*
        gaps.append(gap)
        gpu_ok += gap <= QUALITY
        ora_ok += conv[j]["F"] / fstar[j] - 1.0 <= QUALITY
    slack = math.ceil(0.1 * len(idx))
    print(f"{name}: bf16x2 {gpu_ok}/{len(idx)} within 1e-4 of F*, oracle {ora_ok}/{len(idx)} "
          f"under the same rule; median gap {np.median(gaps):.2e}")
    # plans that sit on the edge of the 1e-4 bar flip either way with the rounding of the
    # path (see the module docstring), hence a slack of 10 % of the sample
    assert gpu_ok >= ora_ok - slack
    return p, W, idx, conv, out


def test_bf16x2_solve_quality_small(gmco_mod, oracle_mod):
    _solve_quality(gmco_mod, oracle_mod, "prostate-2k-8plans", 8)


def test_bf16x2_solve_quality_paper_scale_sample(gmco_mod, oracle_mod):
    _solve_quality(gmco_mod, oracle_mod, "prostate-12k-1000plans", 64)


@pytest.mark.parametrize("name,n", [("prostate-2k-8plans", 8), ("prostate-12k-1000plans", 64)])
def test_converged_dvh_vs_optimum(gmco_mod, oracle_mod, name, n):
    """V100 and D90 of converged bf16x2 plans against those of the exact optimum, within
    0.5 percentage points on at least as many plans as the oracle's own L-BFGS (minus the
    same 10 % slack); the misses are printed.  V100 is fragile at the optimum: many target
    points sit on the prescription there, so plans with objectives 1e-4 apart can differ
    by whole points."""
    p, W, idx, conv, out = _solve_quality(gmco_mod, oracle_mod, name, n)
    gpu_ok = ora_ok = 0
    misses = []
    for r, j in enumerate(idx):
        c = conv[j]
        dv, dd = out["dvh"][r][0] - c["v100_star"], out["dvh"][r][1] - c["d90_star"]
        ok = abs(dv) <= 0.5 and abs(dd) <= 0.5
        gpu_ok += ok
        ora_ok += abs(c["v100"] - c["v100_star"]) <= 0.5 and abs(c["d90"] - c["d90_star"]) <= 0.5
        if not ok:
            misses.append((int(j), round(float(dv), 3), round(float(dd), 3)))
    print(f"{name}: V100/D90 within 0.5 pp of the optimum's: bf16x2 {gpu_ok}/{len(idx)}, "
          f"oracle L-BFGS {ora_ok}/{len(idx)}; misses (plan, dV100, dD90): {misses}")
    assert gpu_ok >= ora_ok - math.ceil(0.1 * len(idx))


@pytest.mark.parametrize("form", ["fp32", "bf16x3"])
@pytest.mark.parametrize("m,k", [(10, 12), (10, 25), (2, 10), (3, 10)])
def test_path_past_history_wrap(gmco_mod, oracle_mod, form, m, k):
    """k accepted iterations with an m-pair history (k > m: the ring has wrapped) against
    the oracle: the same iterations and status, F and T within ten times the oracle's own
    spread.  With m = 2 and 3 the ring wraps several times within 10 iterations, early
    enough for the tolerances to stay tight; a wrong slot order after a wrap changes the
    direction and shows up in F and T far beyond them."""
    p, W, _ = workload("prostate-2k-8plans")
    prm = smooth_params(p.params)
    spread = oracle_self_spread(oracle_mod, p.A, p.sid, prm, W, FORM_EPS[form], max_iters=k,
                                tol=0.0, m=m)
    with gmco_mod.Problem(p.A, p.sid, prm, precision=form, m=m) as pr:
        out = pr.solve_batch(W, max_iters=k, tol=0.0)
    worst = []
    for j in range(W.shape[0]):
        s = spread[j]
        r = s["r"]
        assert out["iters"][j] == r["iters"] == k
        assert out["status"][j] == r["status"] == oracle_mod.MAXITER
        dF = abs(out["objectives"][j] / r["F"] - 1.0)
        dT = float(np.max(np.abs(out["T"][j] - r["t"])) / np.max(np.abs(r["t"])))
        # floors: the forms' own accumulation errors, which a perturbation of A models only in
        # part (FP32 sums over 2000 points, and for bf16x3 its 2.2e-6 dose error)
        tol_F = max(10.0 * s["dF"], FLOOR_F[form])
        tol_T = max(10.0 * s["dT"], FLOOR_T[form])
        worst.append((round(dF / tol_F, 3), round(dT / tol_T, 3)))
        assert dF <= tol_F, (j, dF, s["dF"])
        assert dT <= tol_T, (j, dT, s["dT"])
    print(f"{form} m={m} k={k}: deviation / tolerance per plan (F, T): {worst}")


@pytest.mark.parametrize("window", [1, 3])
def test_stop_window_follows_oracle(gmco_mod, oracle_mod, window):
    """stop_window = 3: a plan stops after three consecutive accepted iterations each within
    the relative tolerance, as the oracle does; the iteration counts equal the oracle's
    wherever the oracle's own perturbed run keeps them, and a window of 3 never stops
    earlier than a window of 1."""
    p, W, _ = workload("prostate-2k-8plans")
    prm = smooth_params(p.params)
    tol = 3e-3
    spread = oracle_self_spread(oracle_mod, p.A, p.sid, prm, W, FORM_EPS["fp32"], max_iters=500,
                                tol=tol, stop_window=window)
    with gmco_mod.Problem(p.A, p.sid, prm, precision="fp32", stop_window=window) as pr:
        out = pr.solve_batch(W, max_iters=500, tol=tol)
    with gmco_mod.Problem(p.A, p.sid, prm, precision="fp32", stop_window=1) as pr1:
        one = pr1.solve_batch(W, max_iters=500, tol=tol)
    stable = 0
    for j in range(W.shape[0]):
        s = spread[j]
        assert out["status"][j] == s["r"]["status"] == oracle_mod.CONVERGED
        assert out["iters"][j] >= one["iters"][j]
        if s["r"]["iters"] == s["r2"]["iters"]:
            stable += 1
            assert out["iters"][j] == s["r"]["iters"], (j, out["iters"][j], s["r"]["iters"])
            assert abs(out["objectives"][j] / s["r"]["F"] - 1.0) <= max(10.0 * s["dF"], 1e-6)
    assert stable >= 4   # the comparison is not empty (8 and 4 plans keep their counts)
    print(f"window {window}: gpu iters {out['iters'].tolist()}, oracle "
          f"{[s['r']['iters'] for s in spread]}")


def test_bf16x2_full_batch_in_bench_configuration(gmco_mod):
    """The headline workload in the benchmark's launch configuration: all 1000 plans in one
    solve under its rule.  Every reported objective is Eq. (obj) at the returned dwell times
    (FP64 oracle) within the FP32 re-evaluation's bound, none falls below its exact optimum F*,
    and the fraction within 1e-4 of F* is at least the oracle L-BFGS's on the golden sample of
    the same workload and rule, less the same 10 % slack."""
    from oracle import optimum
    name = "prostate-12k-1000plans"
    p, W, _ = workload(name)
    fstar = read_fstar(name)
    conv = read_converged(name)
    # the benchmark's options (steps_per_poll 32: the host compacts the live rows every 32 steps,
    # which sets the gradient GEMM's split plan and so the rounding of the path)
    with gmco_mod.Problem(p.A, p.sid, p.params, precision="bf16x2", max_evals=MAX_EVALS,
                          steps_per_poll=32) as pr:
        out = pr.solve_batch(W, allow_timeout=True, **RULE)
    P = W.shape[0]
    ok = 0
    worst = 0.0
    for j in range(P):
        F_o = optimum.objective_t(p.A, p.sid, p.params, W[j], out["T"][j].astype(np.float64))[0]
        dev = abs(out["objectives"][j] / F_o - 1.0)
        worst = max(worst, dev)
        assert dev <= REPORT_TOL[name], (j, out["objectives"][j], F_o)
        gap = F_o / fstar[j] - 1.0
        assert gap >= -1e-9, (j, gap)
        ok += gap <= QUALITY
    ora = sum(c["F"] / c["Fstar"] - 1.0 <= QUALITY for c in conv.values()) / len(conv)
    print(f"full batch: {ok}/{P} within 1e-4 of F*; oracle fraction on its sample {ora:.3f}; "
          f"worst reported-F deviation {worst:.2e}")
    assert ok >= (ora - 0.1) * P
