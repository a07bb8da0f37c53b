"""Exact optimal value F* = min_{t >= 0} F(t) of one plan.  Test infrastructure only.

Eq. (obj) with Eq. (1) and Eq. (dose) is convex in t (a sum of convex piecewise quadratics of
linear functions of t; the paper notes the convex solution space in Sec. 4), so its minimum
over the non-negative orthant has a single value even where the minimiser is not unique.
The L-BFGS method of the paper approaches it slowly (its x = sqrt(t) substitution is badly
conditioned near dwells that switch off), so the reference value the benchmark and the
tests grade against is computed here by a different, exact route:

  repeat:
    1. at the current t, take the set of violated points (d_i < D_min or d_i > D_max),
       each with its bound as target and sqrt(w_s / N_s * w_min|w_max) as row weight;
    2. solve that weighted non-negative least-squares problem exactly
       (Lawson-Hanson, scipy.optimize.nnls, a library routine used as one step);
    3. move from t towards the NNLS solution with an exact line search on the true F
       (convex along the segment, which stays in t >= 0);
  until the violated set stops changing; then certify optimality by the KKT conditions
  of the convex problem (dF/dt_l >= 0 where t_l = 0, dF/dt_l = 0 where t_l > 0).

Everything is float64 numpy; F and its t-gradient are written out from Eq. (1)/(obj).
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import nnls


def _parts(A, sid, params, w):
    A = np.ascontiguousarray(A, dtype=np.float64)
    sid = np.asarray(sid, dtype=np.int64)
    params = np.asarray(params, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    N = np.bincount(sid, minlength=params.shape[0]).astype(np.float64)
    c = np.where(N[sid] > 0, w[sid] / np.maximum(N[sid], 1.0), 0.0)   # w_s / N_s per point
    return A, sid, params, c


def objective_t(A, sid, params, w, t):
    """F(t) of Eq. (obj) and dF/dt (float64)."""
    A, sid, params, c = _parts(A, sid, params, w)
    d = A @ t
    lo, hi = params[sid, 1], params[sid, 2]
    wmin, wmax = params[sid, 0], params[sid, 3]
    under = np.where(d < lo, lo - d, 0.0)
    over = np.where(d > hi, d - hi, 0.0)
    F = float(np.sum(c * (wmin * under ** 2 + wmax * over ** 2)))
    gd = c * (-2.0 * wmin * under + 2.0 * wmax * over)
    return F, A.T @ gd


def kkt_residual(A, sid, params, w, t, t_zero=None):
    """Largest KKT violation of min_{t>=0} F, relative to the gradient's term scale.

    Dwells with t_l <= t_zero (default 1e-6 max(t)) count as switched off: there only a
    negative gradient violates the conditions."""
    A_, sid_, params_, c = _parts(A, sid, params, w)
    F, g = objective_t(A, sid, params, w, t)
    d = A_ @ t
    lo, hi = params_[sid_, 1], params_[sid_, 2]
    wmin, wmax = params_[sid_, 0], params_[sid_, 3]
    gd_abs = np.abs(c * (2.0 * wmin * np.where(d < lo, lo - d, 0.0)
                         + 2.0 * wmax * np.where(d > hi, d - hi, 0.0)))
    scale = float(np.max(A_.T @ gd_abs)) or 1.0
    if t_zero is None:
        t_zero = 1e-6 * float(np.max(t)) if np.max(t) > 0 else 0.0
    pos = t > t_zero
    r_pos = np.max(np.abs(g[pos])) if np.any(pos) else 0.0
    r_zero = np.max(np.maximum(-g[~pos], 0.0)) if np.any(~pos) else 0.0
    return max(r_pos, r_zero) / scale


def _line_search(A, sid, params, w, t, t_new):
    """argmin_{theta in [0,1]} F(t + theta (t_new - t)), by bisection on the derivative."""
    dt = t_new - t

    def dphi(th):
        return float(objective_t(A, sid, params, w, t + th * dt)[1] @ dt)

    if dphi(1.0) <= 0.0:
        return 1.0
    lo, hi = 0.0, 1.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if dphi(mid) > 0.0:
            hi = mid
        else:
            lo = mid
    return lo


def fstar(A, sid, params, w, t_init=None, max_rounds=200):
    """Returns dict(F, t, rounds, kkt): the exact minimum of F over t >= 0."""
    A_, sid_, params_, c = _parts(A, sid, params, w)
    n = A_.shape[1]
    t = np.ones(n) if t_init is None else np.asarray(t_init, dtype=np.float64).copy()
    lo, hi = params_[sid_, 1], params_[sid_, 2]
    wmin, wmax = params_[sid_, 0], params_[sid_, 3]
    prev_key = None
    rounds = 0
    for rounds in range(1, max_rounds + 1):
        d = A_ @ t
        under = d < lo
        over = d > hi
        act = under | over
        key = (under.tobytes(), over.tobytes())
        if key == prev_key:
            break
        prev_key = key
        if not np.any(act):
            break
        target = np.where(under, lo, hi)[act]
        rw = np.sqrt(c[act] * np.where(under, wmin, wmax)[act])
        t_new, _ = nnls(rw[:, None] * A_[act], rw * target, maxiter=50 * n)
        theta = _line_search(A_, sid_, params_, w, t, t_new)
        t = t + theta * (t_new - t)
        t = np.maximum(t, 0.0)
    F, _ = objective_t(A_, sid_, params_, w, t)
    return dict(F=F, t=t, rounds=rounds, kkt=kkt_residual(A_, sid_, params_, w, t))
