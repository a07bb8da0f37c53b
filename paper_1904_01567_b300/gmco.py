"""Thin ctypes binding of libgmco.so (include/gmco.h).  Argument marshalling only.

Functions carry the C names without the ``gmco_`` prefix.  Arrays may be numpy arrays
(host memory) or torch tensors (host or CUDA memory); outputs are allocated where the
inputs live (torch CUDA tensors on the current device, numpy arrays otherwise).  Every
computation runs in the CUDA library: there is no CPU fallback, and a missing or unloadable
library raises at first use.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgmco.so")

PREC = {"fp32": 0, "bf16": 1, "fp8": 2, "bf16x2": 3, "bf16x3": 4}
PLAN_STATUS = {0: "converged", 1: "maxiter", 2: "lsfail", 3: "nonfinite"}
DVH_K = 5
DVH_NAMES = ("V100_pct", "D90_pct_rx", "urethra_D10_pct_rx", "rectum_V75_pct", "bladder_V75_pct")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED = 0, 1, 2, 3, 4, 5


class GmcoError(RuntimeError):
    def __init__(self, status, where, detail=""):
        super().__init__(f"{where}: {status_string(status)} ({status}) {detail}".strip())
        self.status = status


class _Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("m", ctypes.c_int32), ("c1", ctypes.c_double),
                ("max_ls", ctypes.c_int32), ("rx_gy", ctypes.c_double),
                ("refine_iters", ctypes.c_int32), ("steps_per_poll", ctypes.c_int32),
                ("stop_window", ctypes.c_int32), ("grad_split_kb", ctypes.c_int32),
                ("max_evals", ctypes.c_int32), ("grad_plan_tile", ctypes.c_int32),
                ("sparse_grad_permille", ctypes.c_int32), ("wait_limit_us", ctypes.c_int32)]


class _Geometry(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("a", "b", "c", "urethra_r", "rectum_r", "rectum_y",
                                             "rectum_half_len", "bladder_r", "bladder_z")]


class _Source(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("sk", ctypes.c_double), ("unit", ctypes.c_double),
                ("r_min", ctypes.c_double), ("g0", ctypes.c_double), ("g1", ctypes.c_double),
                ("g2", ctypes.c_double)]


class _Rtog(ctypes.Structure):
    _fields_ = [("v100_min", ctypes.c_double), ("v100_min_plus", ctypes.c_double),
                ("d10_max", ctypes.c_double), ("v75_max_cc", ctypes.c_double),
                ("vol_cc", ctypes.c_double * 2)]


class _SaOptions(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("seed", ctypes.c_uint64), ("T0", ctypes.c_double),
                ("T_final", ctypes.c_double), ("step0", ctypes.c_double),
                ("step_final", ctypes.c_double)]


_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32


def load():
    """Loads libgmco.so (built in-tree by paper_1904_01567_b300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run python -m paper_1904_01567_b300.build")
        lib = ctypes.CDLL(LIB_PATH)
        lib.gmco_default_options.argtypes = [ctypes.POINTER(_Options)]
        lib.gmco_default_options.restype = None
        lib.gmco_default_source.argtypes = [ctypes.POINTER(_Source)]
        lib.gmco_default_source.restype = None
        lib.gmco_dose_rate_matrix.argtypes = [_vp, _i64, _vp, _i64, ctypes.POINTER(_Source), _vp, _vp]
        lib.gmco_dose_rate_matrix.restype = ctypes.c_int
        lib.gmco_default_rtog.argtypes = [ctypes.POINTER(_Rtog)]
        lib.gmco_default_rtog.restype = None
        lib.gmco_rtog_select.argtypes = [_vp, _i64, ctypes.POINTER(_Rtog), _vp, _vp, _vp]
        lib.gmco_rtog_select.restype = ctypes.c_int
        lib.gmco_pareto_filter.argtypes = [_vp, _i64, _i32, _vp, _vp]
        lib.gmco_pareto_filter.restype = ctypes.c_int
        lib.gmco_create_problem.argtypes = [_vp, _i64, _i64, _vp, _i32, _vp,
                                            ctypes.POINTER(_Options), ctypes.POINTER(_vp)]
        lib.gmco_create_problem.restype = ctypes.c_int
        lib.gmco_destroy_problem.argtypes = [_vp]
        lib.gmco_destroy_problem.restype = None
        lib.gmco_solve_batch.argtypes = [_vp, _vp, _i64, _vp, _i32, ctypes.c_double, _vp, _vp,
                                         _vp, _vp, _vp, _vp]
        lib.gmco_solve_batch.restype = ctypes.c_int
        lib.gmco_default_sa_options.argtypes = [_vp]
        lib.gmco_default_sa_options.restype = None
        lib.gmco_solve_sa.argtypes = [_vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp]
        lib.gmco_solve_sa.restype = ctypes.c_int
        lib.gmco_evaluate.argtypes = [_vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp]
        lib.gmco_evaluate.restype = ctypes.c_int
        lib.gmco_sample_points.argtypes = [ctypes.POINTER(_Geometry), _vp, ctypes.c_uint64, _vp, _vp, _vp]
        lib.gmco_sample_points.restype = ctypes.c_int
        lib.gmco_fp32_peak.argtypes = [_i32, _i32, _vp]
        lib.gmco_fp32_peak.restype = ctypes.c_int
        lib.gmco_dvh_at.argtypes = [_vp, _vp, _i64, _vp, _vp]
        lib.gmco_dvh_at.restype = ctypes.c_int
        lib.gmco_evaluate_noalloc.argtypes = [_vp, _vp, _i64, _vp, _vp, _vp, _vp]
        lib.gmco_evaluate_noalloc.restype = ctypes.c_int
        lib.gmco_dvh_from_dose.argtypes = [_vp, _vp, _i64, _vp, _vp]
        lib.gmco_dvh_from_dose.restype = ctypes.c_int
        lib.gmco_profile_evaluate.argtypes = [_vp, _vp, _i64, _vp, _i32, _vp, _vp]
        lib.gmco_profile_evaluate.restype = ctypes.c_int
        lib.gmco_problem_info.argtypes = [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                          ctypes.POINTER(_i32), ctypes.POINTER(_i32)]
        lib.gmco_problem_info.restype = ctypes.c_int
        lib.gmco_last_launch_count.argtypes = [_vp]
        lib.gmco_last_launch_count.restype = _i64
        lib.gmco_last_sparse_steps.argtypes = [_vp]
        lib.gmco_last_sparse_steps.restype = _i64
        lib.gmco_status_string.argtypes = [ctypes.c_int]
        lib.gmco_status_string.restype = ctypes.c_char_p
        lib.gmco_last_error.argtypes = []
        lib.gmco_last_error.restype = ctypes.c_char_p
        lib.gmco_create_multi.argtypes = [_vp, _i32, ctypes.POINTER(_vp)]
        lib.gmco_create_multi.restype = ctypes.c_int
        lib.gmco_destroy_multi.argtypes = [_vp]
        lib.gmco_destroy_multi.restype = None
        lib.gmco_multi_set_split.argtypes = [_vp, _i32]
        lib.gmco_multi_set_split.restype = ctypes.c_int
        lib.gmco_multi_get_split.argtypes = [_vp]
        lib.gmco_multi_get_split.restype = _i32
        lib.gmco_multi_set_tiles.argtypes = [_vp, _i32, _i32]
        lib.gmco_multi_set_tiles.restype = ctypes.c_int
        lib.gmco_multi_get_grad_tile.argtypes = [_vp]
        lib.gmco_multi_get_grad_tile.restype = _i32
        lib.gmco_multi_autotune_tiles.argtypes = [_vp, _vp, _vp, _i32, _vp, _vp, _i32, _vp, _vp]
        lib.gmco_multi_autotune_tiles.restype = ctypes.c_int
        lib.gmco_multi_last_launch_count.argtypes = [_vp]
        lib.gmco_multi_last_launch_count.restype = _i64
        lib.gmco_solve_multi.argtypes = [_vp, _vp, _vp, _vp, _i32, ctypes.c_double, _vp, _vp, _vp,
                                         _vp, _vp, _vp]
        lib.gmco_solve_multi.restype = ctypes.c_int
        lib.gmco_multi_autotune.argtypes = [_vp, _vp, _vp, _i32, _vp, _i32, _vp, _vp]
        lib.gmco_multi_autotune.restype = ctypes.c_int
        lib.gmco_mlp_create.argtypes = [_vp, ctypes.POINTER(_vp)]
        lib.gmco_mlp_create.restype = ctypes.c_int
        lib.gmco_mlp_destroy.argtypes = [_vp]
        lib.gmco_mlp_destroy.restype = None
        lib.gmco_mlp_get_params.argtypes = [_vp, _vp]
        lib.gmco_mlp_get_params.restype = ctypes.c_int
        lib.gmco_mlp_save.argtypes = [_vp, ctypes.c_char_p]
        lib.gmco_mlp_save.restype = ctypes.c_int
        lib.gmco_mlp_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(_vp)]
        lib.gmco_mlp_load.restype = ctypes.c_int
        lib.gmco_mlp_predict.argtypes = [_vp, _vp, _i64, _vp, _i64, ctypes.c_float, _vp, _vp]
        lib.gmco_mlp_predict.restype = ctypes.c_int
        lib.gmco_mlp_gradient.argtypes = [_vp, _vp, _i64, _vp, _i64, _vp, _vp, _i64, _vp, _vp, _vp]
        lib.gmco_mlp_gradient.restype = ctypes.c_int
        lib.gmco_mlp_train_step.argtypes = [_vp, _vp, _i64, _vp, _i64, _vp, _vp, _i64,
                                            ctypes.c_float, _vp, _vp]
        lib.gmco_mlp_train_step.restype = ctypes.c_int
        lib.gmco_mlp_last_launch_count.argtypes = [_vp]
        lib.gmco_mlp_last_launch_count.restype = _i64
        lib.gmco_mlp_last_error.argtypes = []
        lib.gmco_mlp_last_error.restype = ctypes.c_char_p
        lib.gmco_warm_start.argtypes = [_vp, _vp, _vp, _vp, _i64, ctypes.c_float, _vp, _vp, _vp]
        lib.gmco_warm_start.restype = ctypes.c_int
        _lib = lib
    return _lib


def status_string(status: int) -> str:
    return load().gmco_status_string(int(status)).decode()


def last_error() -> str:
    return load().gmco_last_error().decode()


def _check(status, where):
    if status != OK:
        raise GmcoError(status, where, last_error())


# ---------------------------------------------------------------- marshalling helpers
def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _prep(a, np_dtype, torch_name):
    """Contiguous array of the right dtype; returns (keepalive, pointer, is_cuda)."""
    if a is None:
        return None, None, False
    if _is_torch(a):
        import torch
        t = a.detach().to(getattr(torch, torch_name)).contiguous()
        return t, t.data_ptr(), t.is_cuda
    arr = np.ascontiguousarray(a, dtype=np_dtype)
    return arr, arr.ctypes.data, False


def _alloc(shape, np_dtype, torch_name, cuda):
    if cuda:
        import torch
        t = torch.empty(shape, dtype=getattr(torch, torch_name), device="cuda")
        return t, t.data_ptr()
    arr = np.empty(shape, dtype=np_dtype)
    return arr, arr.ctypes.data


def _stream_ptr(stream, cuda):
    if stream is not None:
        return int(getattr(stream, "cuda_stream", stream))
    if cuda:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return 0


# ---------------------------------------------------------------- C ABI mirrors
def default_options(**overrides) -> _Options:
    o = _Options()
    load().gmco_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if k == "precision" and isinstance(v, str):
            v = PREC[v]
        setattr(o, k, v)
    return o


def default_source(**overrides) -> _Source:
    """gmco_default_source, with fields replaced by keyword (lambda_, sk, unit, r_min, g0..g2)."""
    s = _Source()
    load().gmco_default_source(ctypes.byref(s))
    for k, v in overrides.items():
        setattr(s, k, v)
    return s


def dose_rate_matrix(points, dwells, source=None, stream=None):
    """gmco_dose_rate_matrix: the n_pnt x n_dwell dose-rate matrix (Gy/s, FP32) of the given
    points and dwell positions (n x 3, cm).  Torch CUDA inputs give a CUDA tensor, else numpy."""
    lib = load()
    p_keep, p_ptr, cuda = _prep(points, np.float32, "float32")
    d_keep, d_ptr, cuda_d = _prep(dwells, np.float32, "float32")
    cuda = cuda or cuda_d
    n_pnt, n_dwell = int(p_keep.shape[0]), int(d_keep.shape[0])
    out, o_ptr = _alloc((n_pnt, n_dwell), np.float32, "float32", cuda)
    src = source if source is not None else default_source()
    _check(lib.gmco_dose_rate_matrix(p_ptr, n_pnt, d_ptr, n_dwell, ctypes.byref(src), o_ptr,
                                     _stream_ptr(stream, cuda)), "gmco_dose_rate_matrix")
    return out


def rtog_select(dvh, rectum_cc, bladder_cc, stream=None, **criteria):
    """gmco_rtog_select: (classes[P] with 2 = RTOG+, 1 = RTOG, 0 = invalid, selected index).
    dvh is P x 5 as solve_batch returns it; criteria override gmco_default_rtog fields."""
    lib = load()
    d_keep, d_ptr, cuda = _prep(dvh, np.float32, "float32")
    P = int(d_keep.shape[0])
    c = _Rtog()
    lib.gmco_default_rtog(ctypes.byref(c))
    for k, v in criteria.items():
        setattr(c, k, v)
    c.vol_cc[0], c.vol_cc[1] = float(rectum_cc), float(bladder_cc)
    cls, c_ptr = _alloc((P,), np.int32, "int32", cuda)
    sel = np.zeros(1, np.int32)
    _check(lib.gmco_rtog_select(d_ptr, P, ctypes.byref(c), c_ptr, sel.ctypes.data,
                                _stream_ptr(stream, cuda)), "gmco_rtog_select")
    return cls, int(sel[0])


def pareto_filter(obj, stream=None):
    """gmco_pareto_filter: 1 for the non-dominated rows of obj (P x K, minimised), else 0."""
    lib = load()
    o_keep, o_ptr, cuda = _prep(obj, np.float64, "float64")
    P, K = int(o_keep.shape[0]), int(o_keep.shape[1])
    out, n_ptr = _alloc((P,), np.int32, "int32", cuda)
    _check(lib.gmco_pareto_filter(o_ptr, P, K, n_ptr, _stream_ptr(stream, cuda)),
           "gmco_pareto_filter")
    return out


def create_problem(A, structure_ids, penalty_params, **options):
    """gmco_create_problem.  Returns an opaque handle (int)."""
    lib = load()
    a_keep, a_ptr, _ = _prep(A, np.float32, "float32")
    s_keep, s_ptr, _ = _prep(structure_ids, np.int32, "int32")
    p_keep, p_ptr, _ = _prep(penalty_params, np.float64, "float64")
    n_pnt, n_dwell = (int(x) for x in a_keep.shape)
    n_struct = int(p_keep.shape[0])
    opt = default_options(**options)
    h = _vp()
    _check(lib.gmco_create_problem(a_ptr, n_pnt, n_dwell, s_ptr, n_struct, p_ptr,
                                   ctypes.byref(opt), ctypes.byref(h)), "gmco_create_problem")
    return h.value


def destroy_problem(h):
    if h:
        load().gmco_destroy_problem(h)


def problem_info(h):
    n_pnt, n_dwell, n_struct, prec = _i64(), _i64(), _i32(), _i32()
    _check(load().gmco_problem_info(h, ctypes.byref(n_pnt), ctypes.byref(n_dwell),
                                    ctypes.byref(n_struct), ctypes.byref(prec)),
           "gmco_problem_info")
    return dict(n_pnt=n_pnt.value, n_dwell=n_dwell.value, n_struct=n_struct.value,
                precision=prec.value)


def last_launch_count(h) -> int:
    return int(load().gmco_last_launch_count(h))


def solve_batch(h, penalty_weights, t0=None, max_iters=500, tol=1e-6, stream=None,
                want=("T", "objectives", "dvh", "iters", "status"), allow_timeout=False):
    """gmco_solve_batch.  Returns a dict with the requested outputs."""
    info = problem_info(h)
    w_keep, w_ptr, cuda = _prep(penalty_weights, np.float32, "float32")
    P = int(w_keep.shape[0])
    t_keep, t_ptr, _ = _prep(t0, np.float32, "float32")
    out, ptrs = {}, {}
    shapes = dict(T=((P, info["n_dwell"]), np.float32, "float32"),
                  objectives=((P,), np.float64, "float64"),
                  dvh=((P, DVH_K), np.float32, "float32"),
                  iters=((P,), np.int32, "int32"), status=((P,), np.int32, "int32"))
    for k in ("T", "objectives", "dvh", "iters", "status"):
        if k in want:
            out[k], ptrs[k] = _alloc(*shapes[k], cuda)
        else:
            ptrs[k] = None
    st = load().gmco_solve_batch(h, w_ptr, P, t_ptr, int(max_iters), float(tol), ptrs["T"],
                                 ptrs["objectives"], ptrs["dvh"], ptrs["iters"], ptrs["status"],
                                 _stream_ptr(stream, cuda))
    if st == ETIMEOUT and allow_timeout:
        out["timeout"] = True
    else:
        _check(st, "gmco_solve_batch")
    del w_keep, t_keep
    return out


def sample_points(geometry, counts, seed, device=False, stream=None):
    """gmco_sample_points: (points (N x 3), sid (N,)) of the analytic structures.  `geometry`
    has the attributes (or keys) a, b, c, urethra_r, rectum_r, rectum_y, rectum_half_len,
    bladder_r, bladder_z (cm); counts: 4 point counts.  device=True returns torch CUDA tensors."""
    get = (lambda k: geometry[k]) if isinstance(geometry, dict) else (lambda k: getattr(geometry, k))
    geo = _Geometry(*[float(get(k)) for k, _ in _Geometry._fields_])
    cnt = np.ascontiguousarray(counts, dtype=np.int64)
    assert cnt.shape == (4,)
    n = int(cnt.sum())
    pts, pptr = _alloc((n, 3), np.float32, "float32", device)
    sid, sptr = _alloc((n,), np.int32, "int32", device)
    _check(load().gmco_sample_points(ctypes.byref(geo), cnt.ctypes.data, ctypes.c_uint64(int(seed) & (2**64 - 1)),
                                     pptr, sptr, _stream_ptr(stream, device)), "gmco_sample_points")
    return pts, sid


def fp32_peak(iters=4096, reps=5):
    """gmco_fp32_peak: (scalar FFMA, paired FP32 FMA) throughput of the current device, TFLOP/s."""
    out = np.zeros(2)
    _check(load().gmco_fp32_peak(int(iters), int(reps), out.ctypes.data), "gmco_fp32_peak")
    return dict(ffma=float(out[0]), ffma2=float(out[1]))


def dvh_at(h, T, stream=None):
    """gmco_dvh_at: DVH indices (P x DVH_K) of dwell times T (P x n_dwell, s) on this problem's
    points, from FP32 doses.  A problem built on a separate, denser point set of the same
    structures and dwell positions gives the DVH of plans optimised on a coarser one."""
    t_keep, t_ptr, cuda = _prep(T, np.float32, "float32")
    P = int(t_keep.shape[0])
    out, optr = _alloc((P, DVH_K), np.float32, "float32", cuda)
    _check(load().gmco_dvh_at(h, t_ptr, P, optr, _stream_ptr(stream, cuda)), "gmco_dvh_at")
    del t_keep
    return out


def default_sa_options(**overrides) -> _SaOptions:
    """gmco_default_sa_options, with fields replaced by keyword (iterations, seed, T0, T_final,
    step0, step_final)."""
    o = _SaOptions()
    load().gmco_default_sa_options(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def solve_sa(h, penalty_weights, t0=None, stream=None, **sa_options):
    """gmco_solve_sa (the annealing engine).  Returns dict(T, objectives, accepts): the best
    dwell times seen, their objectives and the accepted moves of each plan."""
    info = problem_info(h)
    w_keep, w_ptr, cuda = _prep(penalty_weights, np.float32, "float32")
    P = int(w_keep.shape[0])
    t_keep, t_ptr, _ = _prep(t0, np.float32, "float32")
    opt = default_sa_options(**sa_options)
    out, ptrs = {}, {}
    for k, (shape, dt, tdt) in dict(T=((P, info["n_dwell"]), np.float32, "float32"),
                                    objectives=((P,), np.float64, "float64"),
                                    accepts=((P,), np.int32, "int32")).items():
        out[k], ptrs[k] = _alloc(shape, dt, tdt, cuda)
    _check(load().gmco_solve_sa(h, w_ptr, P, t_ptr, ctypes.byref(opt), ptrs["T"],
                                ptrs["objectives"], ptrs["accepts"], _stream_ptr(stream, cuda)),
           "gmco_solve_sa")
    del w_keep, t_keep
    return out


def evaluate(h, penalty_weights, X, objectives=True, grad=True, dose=False, dvh=False,
             stream=None):
    """gmco_evaluate at dwell weights X (P x n_dwell)."""
    info = problem_info(h)
    w_keep, w_ptr, cuda = _prep(penalty_weights, np.float32, "float32")
    x_keep, x_ptr, _ = _prep(X, np.float32, "float32")
    P = int(w_keep.shape[0])
    out, ptrs = {}, {}
    spec = dict(objectives=(objectives, (P,), np.float64, "float64"),
                grad=(grad, (P, info["n_dwell"]), np.float32, "float32"),
                dose=(dose, (P, info["n_pnt"]), np.float32, "float32"),
                dvh=(dvh, (P, DVH_K), np.float32, "float32"))
    for k, (on, shape, nd_, td_) in spec.items():
        if on:
            out[k], ptrs[k] = _alloc(shape, nd_, td_, cuda)
        else:
            ptrs[k] = None
    _check(load().gmco_evaluate(h, w_ptr, P, x_ptr, ptrs["objectives"], ptrs["grad"],
                                ptrs["dose"], ptrs["dvh"], _stream_ptr(stream, cuda)),
           "gmco_evaluate")
    del w_keep, x_keep
    return out


def profile_evaluate(h, penalty_weights, X, reps=20):
    """gmco_profile_evaluate: per-kernel milliseconds of one evaluation and its FLOPs."""
    w_keep, w_ptr, _ = _prep(penalty_weights, np.float32, "float32")
    x_keep, x_ptr, _ = _prep(X, np.float32, "float32")
    ms = np.zeros(4)
    fl = np.zeros(4)
    _check(load().gmco_profile_evaluate(h, w_ptr, int(w_keep.shape[0]), x_ptr, int(reps),
                                        ms.ctypes.data, fl.ctypes.data), "gmco_profile_evaluate")
    del w_keep, x_keep
    return dict(ms=dict(prep=ms[0], dose_gemm=ms[1], grad_gemm=ms[2], finish=ms[3]),
                flops=dict(dose_algorithmic=fl[0], grad_algorithmic=fl[1], dose_issued=fl[2],
                           grad_issued=fl[3]))


def evaluate_noalloc(h, penalty_weights, X, objectives=None, grad=None, stream=None):
    """gmco_evaluate_noalloc: FP32 objectives and gradient without any device allocation in
    the call.  penalty_weights, X and the outputs must be torch CUDA tensors; outputs are
    allocated here (by torch) when not given.  Queued on `stream` (default: torch's current)
    and not waited for."""
    import torch
    info = problem_info(h)
    w = penalty_weights.detach().to(torch.float32).contiguous()
    x = X.detach().to(torch.float32).contiguous()
    P = int(w.shape[0])
    # the C call takes P from here and trusts the row lengths, so every shape is checked
    if tuple(w.shape) != (P, info["n_struct"]):
        raise ValueError(f"penalty_weights must be P x {info['n_struct']}, got {tuple(w.shape)}")
    if tuple(x.shape) != (P, info["n_dwell"]):
        raise ValueError(f"X must be {P} x {info['n_dwell']}, got {tuple(x.shape)}")
    if not (w.is_cuda and x.is_cuda) or w.device != x.device:
        raise ValueError("penalty_weights and X must be CUDA tensors on the problem's device")
    if objectives is None:
        objectives = torch.empty(P, dtype=torch.float64, device=w.device)
    if grad is None:
        grad = torch.empty((P, info["n_dwell"]), dtype=torch.float32, device=w.device)
    if (tuple(objectives.shape) != (P,) or objectives.dtype != torch.float64
            or not objectives.is_contiguous() or objectives.device != w.device):
        raise ValueError("objectives must be a contiguous float64 CUDA tensor of P values")
    if (tuple(grad.shape) != (P, info["n_dwell"]) or grad.dtype != torch.float32
            or not grad.is_contiguous() or grad.device != w.device):
        raise ValueError("grad must be a contiguous float32 CUDA tensor of P x n_dwell")
    _check(load().gmco_evaluate_noalloc(h, w.data_ptr(), P, x.data_ptr(), objectives.data_ptr(),
                                        grad.data_ptr(), _stream_ptr(stream, True)),
           "gmco_evaluate_noalloc")
    return dict(objectives=objectives, grad=grad, _keep=(w, x))


def dvh_from_dose(h, dose, stream=None):
    """gmco_dvh_from_dose: DVH indices of given doses (P x n_pnt)."""
    d_keep, d_ptr, cuda = _prep(dose, np.float32, "float32")
    P = int(d_keep.shape[0])
    out, optr = _alloc((P, DVH_K), np.float32, "float32", cuda)
    _check(load().gmco_dvh_from_dose(h, d_ptr, P, optr, _stream_ptr(stream, cuda)),
           "gmco_dvh_from_dose")
    return out


class Problem:
    """Owning wrapper of a problem handle."""

    def __init__(self, A, structure_ids, penalty_params, **options):
        self.handle = create_problem(A, structure_ids, penalty_params, **options)
        self.info = problem_info(self.handle)

    @classmethod
    def from_geometry(cls, points, structure_ids, dwells, penalty_params, source=None, **options):
        """Step (i) on the device: the dose rate matrix of the points and dwell positions
        (n x 3, cm; gmco_dose_rate_matrix), then the problem created from that device matrix."""
        import torch

        def dev(a):
            if isinstance(a, torch.Tensor):
                return a.detach().to(device="cuda", dtype=torch.float32).contiguous()
            return torch.as_tensor(np.asarray(a, np.float32)).cuda()
        pts, dws = dev(points), dev(dwells)
        A = dose_rate_matrix(pts, dws, source=source)
        torch.cuda.synchronize()
        return cls(A, structure_ids, penalty_params, **options)

    def solve_batch(self, penalty_weights, t0=None, max_iters=500, tol=1e-6, **kw):
        return solve_batch(self.handle, penalty_weights, t0, max_iters, tol, **kw)

    def dvh_at(self, T, **kw):
        return dvh_at(self.handle, T, **kw)

    def solve_sa(self, penalty_weights, t0=None, **kw):
        return solve_sa(self.handle, penalty_weights, t0, **kw)

    def evaluate(self, penalty_weights, X, **kw):
        return evaluate(self.handle, penalty_weights, X, **kw)

    def dvh_from_dose(self, dose, **kw):
        return dvh_from_dose(self.handle, dose, **kw)

    def evaluate_noalloc(self, penalty_weights, X, **kw):
        return evaluate_noalloc(self.handle, penalty_weights, X, **kw)

    def profile_evaluate(self, penalty_weights, X, reps=20):
        return profile_evaluate(self.handle, penalty_weights, X, reps)

    def last_launch_count(self):
        return last_launch_count(self.handle)

    def last_sparse_steps(self):
        """Steps of the last tensor-core solve with the active-set gradient (-1: option off)."""
        return int(load().gmco_last_sparse_steps(self.handle))

    def close(self):
        if self.handle:
            destroy_problem(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- several patients
def _ptr_array(ptrs):
    arr = (_vp * len(ptrs))()
    for i, p in enumerate(ptrs):
        arr[i] = p
    return arr


class Multi:
    """Owning wrapper of gmco_multi: several problems (patients) solved in one launch per
    step.  `problems` are Problem objects that must outlive this object."""

    def __init__(self, problems):
        self.problems = list(problems)
        hs = _ptr_array([pr.handle for pr in self.problems])
        h = _vp()
        _check(load().gmco_create_multi(ctypes.cast(hs, _vp), len(self.problems), ctypes.byref(h)),
               "gmco_create_multi")
        self.handle = h.value

    @property
    def split(self) -> int:
        return int(load().gmco_multi_get_split(self.handle))

    @split.setter
    def split(self, kb: int):
        _check(load().gmco_multi_set_split(self.handle, int(kb)), "gmco_multi_set_split")

    @property
    def tiles(self):
        """(split length in 64-point blocks, plans per gradient-GEMM tile; 0 = default)."""
        return (int(load().gmco_multi_get_split(self.handle)),
                int(load().gmco_multi_get_grad_tile(self.handle)))

    @tiles.setter
    def tiles(self, value):
        kb, tile = value
        _check(load().gmco_multi_set_tiles(self.handle, int(kb), int(tile)), "gmco_multi_set_tiles")

    def last_launch_count(self) -> int:
        return int(load().gmco_multi_last_launch_count(self.handle))

    def _weights(self, weights):
        keeps, ptrs, cuda = [], [], False
        for w in weights:
            k, ptr, c = _prep(w, np.float32, "float32")
            keeps.append(k)
            ptrs.append(ptr)
            cuda = cuda or c
        P = (_i64 * len(keeps))(*[int(k.shape[0]) for k in keeps])
        return keeps, ptrs, P, cuda

    def solve(self, weights, t0=None, max_iters=500, tol=1e-6, stream=None,
              want=("T", "objectives", "dvh", "iters", "status"), allow_timeout=False):
        """gmco_solve_multi.  weights: one P_p x n_struct array per patient.  Returns a list
        (one dict per patient) with the requested outputs."""
        assert len(weights) == len(self.problems)
        keeps, wptrs, P, cuda = self._weights(weights)
        t_keeps, t_ptrs = [], []
        if t0 is not None:
            for t in t0:
                k, ptr, _ = _prep(t, np.float32, "float32")
                t_keeps.append(k)
                t_ptrs.append(ptr)
        outs = [dict() for _ in self.problems]
        arrays = {}
        for k in ("T", "objectives", "dvh", "iters", "status"):
            if k not in want:
                arrays[k] = None
                continue
            ptrs = []
            for i, pr in enumerate(self.problems):
                n = int(P[i])
                shape, nd_, td_ = dict(T=((n, pr.info["n_dwell"]), np.float32, "float32"),
                                       objectives=((n,), np.float64, "float64"),
                                       dvh=((n, DVH_K), np.float32, "float32"),
                                       iters=((n,), np.int32, "int32"),
                                       status=((n,), np.int32, "int32"))[k]
                outs[i][k], ptr = _alloc(shape, nd_, td_, cuda)
                ptrs.append(ptr)
            arrays[k] = _ptr_array(ptrs)
        wa = _ptr_array(wptrs)
        ta = _ptr_array(t_ptrs) if t0 is not None else None

        def cp(a):
            return ctypes.cast(a, _vp) if a is not None else None
        st = load().gmco_solve_multi(self.handle, cp(wa), ctypes.cast(P, _vp), cp(ta),
                                     int(max_iters), float(tol), cp(arrays["T"]),
                                     cp(arrays["objectives"]), cp(arrays["dvh"]),
                                     cp(arrays["iters"]), cp(arrays["status"]),
                                     _stream_ptr(stream, cuda))
        if st == ETIMEOUT and allow_timeout:
            for o in outs:
                o["timeout"] = True
        else:
            _check(st, "gmco_solve_multi")
        del keeps, t_keeps
        return outs

    def autotune(self, weights, steps=8, candidates=(0, 4, 8, 16, 32, 64)):
        """gmco_multi_autotune: times `steps` solver steps per candidate split length and
        keeps the fastest.  Returns (best, {candidate: ms per step})."""
        keeps, wptrs, P, _ = self._weights(weights)
        cand = (_i32 * len(candidates))(*[int(c) for c in candidates])
        ms = np.zeros(len(candidates))
        best = _i32()
        wa = _ptr_array(wptrs)
        _check(load().gmco_multi_autotune(self.handle, ctypes.cast(wa, _vp), ctypes.cast(P, _vp),
                                          int(steps), ctypes.cast(cand, _vp), len(candidates),
                                          ms.ctypes.data, ctypes.byref(best)),
               "gmco_multi_autotune")
        del keeps
        return int(best.value), {int(c): float(v) for c, v in zip(candidates, ms)}

    def autotune_tiles(self, weights, steps=8, candidates=((0, 0), (16, 0), (32, 0), (32, 128))):
        """gmco_multi_autotune_tiles: candidates are (split length, plans per gradient-GEMM
        tile) pairs; keeps the fastest.  Returns (best pair, {pair: ms per step})."""
        keeps, wptrs, P, _ = self._weights(weights)
        kb = (_i32 * len(candidates))(*[int(c[0]) for c in candidates])
        tl = (_i32 * len(candidates))(*[int(c[1]) for c in candidates])
        ms = np.zeros(len(candidates))
        best = _i32()
        wa = _ptr_array(wptrs)
        _check(load().gmco_multi_autotune_tiles(self.handle, ctypes.cast(wa, _vp), ctypes.cast(P, _vp),
                                                int(steps), ctypes.cast(kb, _vp), ctypes.cast(tl, _vp),
                                                len(candidates), ms.ctypes.data, ctypes.byref(best)),
               "gmco_multi_autotune_tiles")
        del keeps
        pairs = [(int(c[0]), int(c[1])) for c in candidates]
        return pairs[int(best.value)], {p: float(v) for p, v in zip(pairs, ms)}

    def close(self):
        if self.handle:
            load().gmco_destroy_multi(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- learned warm start
MLP_NPARAM = 35073
MLP_NFEAT = 10


def _check_mlp(status, where):
    if status != OK:
        raise GmcoError(status, where, load().gmco_mlp_last_error().decode())


class Mlp:
    """Owning wrapper of gmco_mlp (per-dwell warm-start network).  `params`: the
    GMCO_MLP_NPARAM initial parameters (see include/gmco.h for the layout)."""

    def __init__(self, params=None, handle=None):
        if handle is not None:
            self.handle = handle
            return
        keep, ptr, _ = _prep(params, np.float32, "float32")
        assert int(np.prod(keep.shape)) == MLP_NPARAM
        h = _vp()
        _check_mlp(load().gmco_mlp_create(ptr, ctypes.byref(h)), "gmco_mlp_create")
        self.handle = h.value

    def save(self, path):
        """gmco_mlp_save: parameters, Adam moments and step count to `path`."""
        _check_mlp(load().gmco_mlp_save(self.handle, os.fsencode(path)), "gmco_mlp_save")

    @classmethod
    def load(cls, path):
        """gmco_mlp_load: a network restored from a checkpoint written by save()."""
        h = _vp()
        _check_mlp(load().gmco_mlp_load(os.fsencode(path), ctypes.byref(h)), "gmco_mlp_load")
        return cls(handle=h.value)

    def params(self):
        out = np.empty(MLP_NPARAM, np.float32)
        _check_mlp(load().gmco_mlp_get_params(self.handle, out.ctypes.data), "gmco_mlp_get_params")
        return out

    def last_launch_count(self) -> int:
        return int(load().gmco_mlp_last_launch_count(self.handle))

    def predict(self, features, penalty_weights, t_floor=0.0, stream=None):
        f_keep, f_ptr, cuda = _prep(features, np.float32, "float32")
        w_keep, w_ptr, c2 = _prep(penalty_weights, np.float32, "float32")
        cuda = cuda or c2
        nd, P = int(f_keep.shape[0]), int(w_keep.shape[0])
        out, optr = _alloc((P, nd), np.float32, "float32", cuda)
        _check_mlp(load().gmco_mlp_predict(self.handle, f_ptr, nd, w_ptr, P, float(t_floor), optr,
                                           _stream_ptr(stream, cuda)), "gmco_mlp_predict")
        del f_keep, w_keep
        return out

    def _batch(self, features, penalty_weights, pairs, target):
        f = _prep(features, np.float32, "float32")
        w = _prep(penalty_weights, np.float32, "float32")
        pr = _prep(pairs, np.int32, "int32")
        tg = _prep(target, np.float32, "float32")
        cuda = f[2] or w[2] or pr[2] or tg[2]
        return (f, w, pr, tg), cuda

    def gradient(self, features, penalty_weights, pairs, target, stream=None):
        (f, w, pr, tg), cuda = self._batch(features, penalty_weights, pairs, target)
        grad = np.empty(MLP_NPARAM, np.float32)
        loss = ctypes.c_float()
        _check_mlp(load().gmco_mlp_gradient(self.handle, f[1], int(f[0].shape[0]), w[1],
                                            int(w[0].shape[0]), pr[1], tg[1], int(tg[0].shape[0]),
                                            ctypes.byref(loss), grad.ctypes.data,
                                            _stream_ptr(stream, cuda)), "gmco_mlp_gradient")
        return float(loss.value), grad

    def train_step(self, features, penalty_weights, pairs, target, lr=1e-3, stream=None):
        (f, w, pr, tg), cuda = self._batch(features, penalty_weights, pairs, target)
        loss = ctypes.c_float()
        _check_mlp(load().gmco_mlp_train_step(self.handle, f[1], int(f[0].shape[0]), w[1],
                                              int(w[0].shape[0]), pr[1], tg[1],
                                              int(tg[0].shape[0]), float(lr), ctypes.byref(loss),
                                              _stream_ptr(stream, cuda)), "gmco_mlp_train_step")
        return float(loss.value)

    def close(self):
        if self.handle:
            load().gmco_mlp_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def warm_start(problem, mlp, features, penalty_weights, t_floor=0.3, stream=None):
    """gmco_warm_start: per-plan start times (model prediction, or uniform where the
    prediction's objective is larger) and the per-plan choice (1 = model)."""
    f_keep, f_ptr, c1 = _prep(features, np.float32, "float32")
    w_keep, w_ptr, c2 = _prep(penalty_weights, np.float32, "float32")
    cuda = c1 or c2
    P = int(w_keep.shape[0])
    t0, tptr = _alloc((P, problem.info["n_dwell"]), np.float32, "float32", cuda)
    flag, fptr = _alloc((P,), np.int32, "int32", cuda)
    _check(load().gmco_warm_start(problem.handle, mlp.handle, f_ptr, w_ptr, P, float(t_floor), tptr,
                                  fptr, _stream_ptr(stream, cuda)), "gmco_warm_start")
    del f_keep, w_keep
    return t0, flag
