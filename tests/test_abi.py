"""The C ABI library: loads, exports every declared entry point, validates on the host."""
import ctypes
import os
import re

import numpy as np
import pytest

from tests.conftest import ROOT


def _declared():
    txt = open(os.path.join(ROOT, "include", "gmco.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gmco_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(gmco_mod):
    lib = ctypes.CDLL(gmco_mod.LIB_PATH)
    names = _declared()
    assert "gmco_solve_batch" in names and "gmco_create_problem" in names
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(gmco_mod):
    assert gmco_mod.status_string(0) == "ok"
    assert "invalid" in gmco_mod.status_string(1)
    assert gmco_mod.status_string(99) == "unknown status"


def test_host_validation_before_device_use(gmco_mod):
    # rejected on the host before any CUDA call: zero dwells, ids out of range
    A = np.ones((4, 3), np.float32)
    prm = np.array([[1.0, 15.0, np.inf, 1.0]])
    with pytest.raises(gmco_mod.GmcoError) as e:
        gmco_mod.create_problem(np.ones((4, 0), np.float32), np.zeros(4, np.int32), prm)
    assert e.value.status == 1


def test_planning_steps_host_validation(gmco_mod):
    """Dose rate matrix, plan selection and non-dominated filter: defaults, and bad sizes or
    constants refused on the host before any device use (so also without a device)."""
    s = gmco_mod.default_source()
    assert (s.lambda_, s.sk, s.r_min, s.g0, s.g1, s.g2) == (1.109, 40700.0, 0.1, 1.0, 0.005, -0.002)
    assert s.unit == pytest.approx(1.0 / 360000.0)
    pts, dws = np.zeros((4, 3), np.float32), np.zeros((2, 3), np.float32)
    for bad in ((pts, np.zeros((0, 3), np.float32), None), (pts, np.zeros((1025, 3), np.float32), None),
                (pts, dws, gmco_mod.default_source(r_min=0.0)),
                (pts, dws, gmco_mod.default_source(lambda_=float("nan")))):
        with pytest.raises(gmco_mod.GmcoError) as e:
            gmco_mod.dose_rate_matrix(bad[0], bad[1], source=bad[2])
        assert e.value.status == gmco_mod.EINVAL
    with pytest.raises(gmco_mod.GmcoError) as e:
        gmco_mod.rtog_select(np.zeros((3, 5), np.float32), -1.0, 10.0)   # negative volume
    assert e.value.status == gmco_mod.EINVAL
    with pytest.raises(gmco_mod.GmcoError) as e:
        gmco_mod.pareto_filter(np.zeros((3, 17)))                          # more than 16 objectives
    assert e.value.status == gmco_mod.EINVAL


def test_options_defaults(gmco_mod):
    o = gmco_mod.default_options()
    assert (o.precision, o.m, o.c1, o.max_ls, o.rx_gy) == (0, 10, 1e-4, 30, 15.0)
    assert gmco_mod.default_options(precision="bf16").precision == 1
    prm = np.array([[1.0, 15.0, np.inf, 1.0]])
    assert o.wait_limit_us == 1000000                       # 1 s
    for bad in (dict(max_evals=-1), dict(grad_plan_tile=64), dict(sparse_grad_permille=-1),
                dict(sparse_grad_permille=1001), dict(wait_limit_us=0),
                dict(wait_limit_us=60000001)):   # rejected before any device use
        with pytest.raises(gmco_mod.GmcoError) as e:
            gmco_mod.create_problem(np.ones((4, 3), np.float32), np.zeros(4, np.int32), prm, **bad)
        assert e.value.status == gmco_mod.EINVAL


def test_no_cpu_fallback_without_device(gmco_mod):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(gmco_mod.GmcoError) as e:
        gmco_mod.create_problem(np.ones((4, 3), np.float32), np.zeros(4, np.int32),
                                np.array([[1.0, 15.0, np.inf, 1.0]]))
    assert e.value.status == 3   # GMCO_ECUDA: the library never computes on the host


def test_multi_host_validation(gmco_mod):
    lib = gmco_mod.load()
    h = ctypes.c_void_p()
    assert lib.gmco_create_multi(None, 0, ctypes.byref(h)) == gmco_mod.EINVAL
    assert h.value is None
    arr = (ctypes.c_void_p * 1)(None)
    assert lib.gmco_create_multi(ctypes.cast(arr, ctypes.c_void_p), 1, ctypes.byref(h)) == gmco_mod.EINVAL
    assert lib.gmco_create_multi(ctypes.cast(arr, ctypes.c_void_p), 65, ctypes.byref(h)) == gmco_mod.EINVAL
    assert lib.gmco_multi_set_split(None, 4) == gmco_mod.EINVAL
    assert lib.gmco_multi_get_split(None) == -1
    assert lib.gmco_multi_set_tiles(None, 4, 128) == gmco_mod.EINVAL
    assert lib.gmco_multi_get_grad_tile(None) == -1
    assert lib.gmco_multi_last_launch_count(None) == -1
    lib.gmco_destroy_multi(None)
    assert lib.gmco_solve_multi(None, None, None, None, 1, 0.0, None, None, None, None, None,
                                None) == gmco_mod.EINVAL
    o = gmco_mod.default_options()
    assert o.grad_split_kb == 0 and o.stop_window == 1
    assert o.max_evals == 0 and o.grad_plan_tile == 0 and o.sparse_grad_permille == 0


def test_annealing_options_and_host_validation(gmco_mod):
    """gmco_default_sa_options fills the documented defaults; gmco_solve_sa refuses a missing
    problem or options before any device use."""
    import ctypes
    o = gmco_mod.default_sa_options()
    assert (o.iterations, o.seed, o.T0, o.T_final, o.step0, o.step_final) == (1000, 1, 1e-2, 1e-5, 0.2, 2e-3)
    o2 = gmco_mod.default_sa_options(iterations=5, seed=2**64 - 1)
    assert o2.iterations == 5 and o2.seed == 2**64 - 1
    lib = gmco_mod.load()
    w = (ctypes.c_float * 4)(1, 1, 1, 1)
    assert lib.gmco_solve_sa(None, w, 1, None, ctypes.byref(o), None, None, None, None) == gmco_mod.EINVAL
    assert lib.gmco_solve_sa(None, w, 1, None, None, None, None, None, None) == gmco_mod.EINVAL


def test_mlp_checkpoint_refused_before_device_use(gmco_mod, tmp_path):
    """gmco_mlp_load checks the file (magic line, format version, parameter count, size, finite
    values) before any device use: malformed checkpoints give GMCO_EINVAL with or without a GPU."""
    import ctypes
    lib = gmco_mod.load()
    h = ctypes.c_void_p()
    assert lib.gmco_mlp_load(str(tmp_path / "missing.bin").encode(), ctypes.byref(h)) == gmco_mod.EINVAL
    n = gmco_mod.MLP_NPARAM
    good_hdr = ('{"format": "gmco-mlp", "version": 1, "nparam": %d, "step": 3, "dtype": "float32-le"}\n' % n)
    body = np.zeros(3 * n, np.float32)
    cases = {
        "magic": b"NOT-MLP\n" + good_hdr.encode() + body.tobytes(),
        "version": b"GMCO-MLP\n" + good_hdr.replace('"version": 1', '"version": 2').encode() + body.tobytes(),
        "nparam": b"GMCO-MLP\n" + good_hdr.replace(str(n), str(n - 1)).encode() + body.tobytes(),
        "short": b"GMCO-MLP\n" + good_hdr.encode() + body[:-1].tobytes(),
        "long": b"GMCO-MLP\n" + good_hdr.encode() + body.tobytes() + b"\0",
        "nan": b"GMCO-MLP\n" + good_hdr.encode() + np.where(np.arange(3 * n) == 7, np.nan, 0).astype(np.float32).tobytes(),
        "neg_v": b"GMCO-MLP\n" + good_hdr.encode() + np.where(np.arange(3 * n) == 2 * n + 1, -1.0, 0).astype(np.float32).tobytes(),
    }
    for name, data in cases.items():
        path = tmp_path / f"{name}.bin"
        path.write_bytes(data)
        assert lib.gmco_mlp_load(str(path).encode(), ctypes.byref(h)) == gmco_mod.EINVAL, name
        assert h.value is None
    assert lib.gmco_mlp_save(None, str(tmp_path / "x.bin").encode()) == gmco_mod.EINVAL
