"""ctypes wrapper of the FP64 C oracle (oracle.c).  Test infrastructure only.

Every function takes and returns numpy float64 / int32 arrays; inputs are converted with
np.ascontiguousarray so callers may pass float32 (the values are widened exactly).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

CONVERGED, MAXITER, LSFAIL, NONFINITE = 0, 1, 2, 3

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_lp = ctypes.POINTER(ctypes.c_int64)
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_f64 = ctypes.c_double


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain -O2, OpenMP over plans)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


def load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.oracle_dose.argtypes = [_dp, _i64, _i64, _dp, _dp]
        lib.oracle_dose.restype = None
        lib.oracle_dose_rate.argtypes = [_dp, _i64, _dp, _i64, _dp, _dp]
        lib.oracle_dose_rate.restype = ctypes.c_int
        lib.oracle_rtog_select.argtypes = [_dp, _i64, _dp, _ip, _ip]
        lib.oracle_rtog_select.restype = ctypes.c_int
        lib.oracle_pareto.argtypes = [_dp, _i64, _i32, _ip]
        lib.oracle_pareto.restype = ctypes.c_int
        lib.oracle_point_penalty.argtypes = [_f64, _dp]
        lib.oracle_point_penalty.restype = _f64
        lib.oracle_point_dpenalty.argtypes = [_f64, _dp]
        lib.oracle_point_dpenalty.restype = _f64
        lib.oracle_objective.argtypes = [_dp, _i64, _i64, _ip, _i32, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        lib.oracle_objective.restype = ctypes.c_int
        lib.oracle_two_loop.argtypes = [_i64, _i32, _i32, _i32, _dp, _dp, _dp, _dp, _dp]
        lib.oracle_two_loop.restype = None
        lib.oracle_lbfgs.argtypes = [_dp, _i64, _i64, _ip, _i32, _dp, _dp, _dp, _i32, _f64, _i32,
                                     _f64, _i32, _i32, _i32, _dp, _dp, _ip, _ip, _dp, _lp]
        lib.oracle_lbfgs.restype = ctypes.c_int
        lib.oracle_lbfgs_batch.argtypes = [_dp, _i64, _i64, _ip, _i32, _dp, _dp, _i64, _dp, _i32,
                                           _f64, _i32, _f64, _i32, _i32, _i32, _dp, _dp, _ip, _ip,
                                           _lp, _i32]
        lib.oracle_lbfgs_batch.restype = ctypes.c_int
        lib.oracle_dvh.argtypes = [_dp, _ip, _i64, _i32, _f64, _dp]
        lib.oracle_dvh.restype = None
        _u64 = ctypes.c_uint64
        lib.oracle_splitmix64.argtypes = [_u64, _u64]
        lib.oracle_splitmix64.restype = _u64
        lib.oracle_sa.argtypes = [_dp, _i64, _i64, _ip, _i32, _dp, _dp, _dp, _i64, _i32, _u64,
                                  _f64, _f64, _f64, _f64, _dp, _dp, _ip, _dp, _dp]
        lib.oracle_sa.restype = ctypes.c_int
        lib.oracle_sa_batch.argtypes = [_dp, _i64, _i64, _ip, _i32, _dp, _dp, _i64, _dp, _i32, _u64,
                                        _f64, _f64, _f64, _f64, _dp, _dp, _ip, _dp, _i32]
        lib.oracle_sa_batch.restype = ctypes.c_int
        _lib = lib
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a, t=_dp):
    return None if a is None else a.ctypes.data_as(t)


# the workload's point-source constants: Lambda (cGy h^-1 U^-1), S_K (U), cGy/h -> Gy/s,
# r_min (cm), g(r) = g0 + g1 r + g2 r^2
DEFAULT_SOURCE = (1.109, 40700.0, 1.0 / 360000.0, 0.1, 1.0, 0.005, -0.002)


def dose_rate(points, dwells, source=DEFAULT_SOURCE):
    """Dose rate matrix (n_pnt x n_dwell, Gy/s) of the isotropic point source."""
    pts = _d(points).reshape(-1, 3); dw = _d(dwells).reshape(-1, 3); src = _d(source)
    out = np.empty((pts.shape[0], dw.shape[0]))
    if load().oracle_dose_rate(_p(pts), pts.shape[0], _p(dw), dw.shape[0], _p(src), _p(out)) != 0:
        raise ValueError("oracle_dose_rate: invalid arguments or g(r) <= 0")
    return out


# the RTOG 0924 values of the plan evaluation: V100 >= 90 % (RTOG+ 95 %), urethra D10 < 118 %,
# rectum and bladder V75 < 1 cc
RTOG = (90.0, 95.0, 118.0, 1.0)


def rtog_select(dvh, rectum_cc, bladder_cc, crit=RTOG):
    """(classes, selected index) of a pool's DVH rows (P x 5)."""
    d = _d(dvh).reshape(-1, 5)
    c = _d(list(crit) + [rectum_cc, bladder_cc])
    cls = np.empty(d.shape[0], np.int32)
    sel = np.zeros(1, np.int32)
    if load().oracle_rtog_select(_p(d), d.shape[0], _p(c), _p(cls, _ip), _p(sel, _ip)) != 0:
        raise ValueError("oracle_rtog_select: invalid arguments")
    return cls, int(sel[0])


def pareto(obj):
    """Non-dominated flags (1 / 0) of the rows of obj (P x K, minimised)."""
    o = _d(obj)
    o = o.reshape(o.shape[0], -1)
    out = np.empty(o.shape[0], np.int32)
    if load().oracle_pareto(_p(o), o.shape[0], o.shape[1], _p(out, _ip)) != 0:
        raise ValueError("oracle_pareto: invalid arguments")
    return out


def dose(A, t):
    A = _d(A); t = _d(t)
    out = np.empty(A.shape[0])
    load().oracle_dose(_p(A), A.shape[0], A.shape[1], _p(t), _p(out))
    return out


def point_penalty(d, prm):
    return load().oracle_point_penalty(float(d), _p(_d(prm)))


def point_dpenalty(d, prm):
    return load().oracle_point_dpenalty(float(d), _p(_d(prm)))


def objective(A, sid, params, w, x, want_grad=True):
    """Returns (F, grad_x, dose, f_struct)."""
    A = _d(A); sid = _i(sid); params = _d(params); w = _d(w); x = _d(x)
    S = params.shape[0]
    F = np.zeros(1)
    g = np.empty(A.shape[1]) if want_grad else None
    dd = np.empty(A.shape[0])
    fs = np.empty(S)
    rc = load().oracle_objective(_p(A), A.shape[0], A.shape[1], _p(sid, _ip), S, _p(params),
                                 _p(w), _p(x), _p(F), _p(g), _p(dd), _p(fs))
    if rc != 0:
        raise ValueError("oracle_objective: invalid arguments")
    return float(F[0]), g, dd, fs


def two_loop(S, Y, rho, count, newest, g):
    S = _d(S); Y = _d(Y); rho = _d(rho); g = _d(g)
    m, n = S.shape
    p = np.empty(n)
    load().oracle_two_loop(n, m, count, newest, _p(S), _p(Y), _p(rho), _p(g), _p(p))
    return p


def lbfgs(A, sid, params, w, t0=None, max_iters=200, tol=1e-6, m=10, c1=1e-4, max_ls=30,
          trace=False, stop_window=1, max_evals=0):
    """One plan.  Returns dict(t, F, iters, status, evals[, trace]).  max_evals > 0 caps the
    objective evaluations (the first one and every line-search trial)."""
    A = _d(A); sid = _i(sid); params = _d(params); w = _d(w)
    t0 = None if t0 is None else _d(t0)
    n = A.shape[1]
    t = np.empty(n); F = np.zeros(1); it = np.zeros(1, np.int32); st = np.zeros(1, np.int32)
    ev = np.zeros(1, np.int64)
    tr = np.full(3 * (max_iters + 1), np.nan) if trace else None
    rc = load().oracle_lbfgs(_p(A), A.shape[0], n, _p(sid, _ip), params.shape[0], _p(params),
                             _p(w), _p(t0), max_iters, tol, m, c1, max_ls, stop_window, int(max_evals),
                             _p(t), _p(F), _p(it, _ip), _p(st, _ip), _p(tr), _p(ev, _lp))
    if rc != 0:
        raise ValueError("oracle_lbfgs: invalid arguments")
    out = dict(t=t, F=float(F[0]), iters=int(it[0]), status=int(st[0]), evals=int(ev[0]))
    if trace:
        k = out["iters"]
        out["trace"] = tr.reshape(-1, 3)[:k + 1]
    return out


def lbfgs_batch(A, sid, params, W, T0=None, max_iters=200, tol=1e-6, m=10, c1=1e-4, max_ls=30,
                n_threads=0, stop_window=1, max_evals=0):
    """P plans, one per OpenMP thread.  Returns dict(T, F, iters, status, evals)."""
    A = _d(A); sid = _i(sid); params = _d(params); W = _d(W)
    P = W.shape[0]
    n = A.shape[1]
    T0 = None if T0 is None else _d(T0)
    T = np.empty((P, n)); F = np.empty(P); it = np.empty(P, np.int32); st = np.empty(P, np.int32)
    ev = np.empty(P, np.int64)
    rc = load().oracle_lbfgs_batch(_p(A), A.shape[0], n, _p(sid, _ip), params.shape[0],
                                   _p(params), _p(W), P, _p(T0), max_iters, tol, m, c1, max_ls,
                                   stop_window, int(max_evals), _p(T), _p(F), _p(it, _ip), _p(st, _ip),
                                   _p(ev, _lp), int(n_threads))
    if rc != 0:
        raise ValueError("oracle_lbfgs_batch: invalid arguments")
    return dict(T=T, F=F, iters=it, status=st, evals=ev)


def splitmix64(seed, n):
    """Output n (0-based) of SplitMix64 seeded with `seed`."""
    return int(load().oracle_splitmix64(int(seed) & (2**64 - 1), int(n) & (2**64 - 1)))


def sa(A, sid, params, w, t0=None, iters=1000, seed=1, T0=1e-2, T_final=1e-5, step0=0.2,
       step_final=2e-3, plan=0, trace=False):
    """One plan of the annealing engine (plan = its index in the batch, which keys its draws).
    Returns dict(t, F, accepts, min_margin[, trace])."""
    A = _d(A); sid = _i(sid); params = _d(params); w = _d(w)
    t0 = None if t0 is None else _d(t0)
    n = A.shape[1]
    t = np.empty(n); F = np.zeros(1); acc = np.zeros(1, np.int32); mm = np.zeros(1)
    tr = np.full(iters + 1, np.nan) if trace else None
    rc = load().oracle_sa(_p(A), A.shape[0], n, _p(sid, _ip), params.shape[0], _p(params), _p(w),
                          _p(t0), int(plan), int(iters), int(seed), T0, T_final, step0, step_final,
                          _p(t), _p(F), _p(acc, _ip), _p(mm), _p(tr))
    if rc != 0:
        raise ValueError("oracle_sa: invalid arguments")
    out = dict(t=t, F=float(F[0]), accepts=int(acc[0]), min_margin=float(mm[0]))
    if trace:
        out["trace"] = tr
    return out


def sa_batch(A, sid, params, W, T0s=None, iters=1000, seed=1, T0=1e-2, T_final=1e-5, step0=0.2,
             step_final=2e-3, n_threads=0):
    """P plans of the annealing engine.  Returns dict(T, F, accepts, min_margin)."""
    A = _d(A); sid = _i(sid); params = _d(params); W = _d(W)
    P = W.shape[0]
    n = A.shape[1]
    T0s = None if T0s is None else _d(T0s)
    T = np.empty((P, n)); F = np.empty(P); acc = np.empty(P, np.int32); mm = np.empty(P)
    rc = load().oracle_sa_batch(_p(A), A.shape[0], n, _p(sid, _ip), params.shape[0], _p(params),
                                _p(W), P, _p(T0s), int(iters), int(seed), T0, T_final, step0,
                                step_final, _p(T), _p(F), _p(acc, _ip), _p(mm), int(n_threads))
    if rc != 0:
        raise ValueError("oracle_sa_batch: invalid arguments")
    return dict(T=T, F=F, accepts=acc, min_margin=mm)


def dvh(d, sid, n_struct=4, rx=15.0):
    d = _d(d); sid = _i(sid)
    out = np.empty(5)
    load().oracle_dvh(_p(d), _p(sid, _ip), d.shape[0], n_struct, rx, _p(out))
    return out
