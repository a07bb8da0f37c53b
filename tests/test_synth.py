"""Seeded input generator: sizes, membership, determinism and the dose-rate closed form."""
import numpy as np
import pytest

from synth import (Geometry, dose_rate_matrix, make_patient, weights_dirichlet,
                   weights_loguniform, workload)
from synth.patient import multi_patient_specs


def test_point_source_closed_form():
    # A = Lambda S_K g(r) / r^2 / 360000 Gy/s, values worked by hand:
    # r = 1 cm: 1.109 * 40700 * 1.003 / 360000 = 0.125754747...
    # r = 0.1 cm: 45136.3 * 1.00048 / 0.01 / 360000 = 12.5438793...
    # r = 0.05 cm is clamped to 0.1 cm
    # r = 2 cm: 45136.3 * 1.002 / 4 / 360000 = 0.0314073421...
    # r = 5 cm: 45136.3 * 0.975 / 25 / 360000 = 0.00488976583...
    pts = np.array([[0.05, 0, 0], [0.1, 0, 0], [0, 0.5, 0], [0, 0, 1.0], [2.0, 0, 0], [0, 5.0, 0]])
    A = dose_rate_matrix(pts, np.zeros((1, 3)))[:, 0]
    expect = {0: 12.5438793, 1: 12.5438793, 3: 0.125754747, 4: 0.0314073421, 5: 0.00488976583}
    for i, v in expect.items():
        assert A[i] == pytest.approx(v, rel=2e-6)
    # r = 0.5: g = 1 + 0.0025 - 0.0005 = 1.002 -> 45136.3 * 1.002 / 0.25 / 360000
    assert A[2] == pytest.approx(45136.3 * 1.002 / 0.25 / 360000, rel=1e-12)


def test_membership_and_sizes():
    p = make_patient(123, n_catheters=12, dwell_step=0.5, n_points=(120, 20, 30, 30))
    g = p.geometry
    assert p.points.shape == (200, 3) and p.n_pnt == 200
    assert list(p.n_per_struct) == [120, 20, 30, 30]
    pro = p.points[p.sid == 0]
    assert np.all(g.in_prostate(pro)) and not np.any(g.in_urethra(pro))
    assert np.all(g.in_urethra(p.points[p.sid == 1]))
    rec = p.points[p.sid == 2]
    assert np.all(g.in_rectum(rec)) and not np.any(g.in_prostate(rec))
    bla = p.points[p.sid == 3]
    assert np.all(g.in_bladder(bla)) and not np.any(g.in_prostate(bla) | g.in_rectum(bla))
    # 12 catheters x 8 dwell positions over |z| <= 1.75 cm at 0.5 cm
    assert p.n_dwell == 96
    assert np.all(np.abs(p.dwells[:, 2]) <= g.c + 1e-12)
    assert p.A.dtype == np.float32 and np.all(p.A > 0)


def test_deterministic():
    a = make_patient(7, 12, 0.5, (50, 10, 10, 10))
    b = make_patient(7, 12, 0.5, (50, 10, 10, 10))
    assert np.array_equal(a.A, b.A) and np.array_equal(a.sid, b.sid)
    c = make_patient(8, 12, 0.5, (50, 10, 10, 10))
    assert not np.array_equal(a.points, c.points)


def test_weights():
    w = weights_loguniform(5, 1000)
    assert w.shape == (1000, 4) and w.min() >= 0.1 - 1e-6 and w.max() <= 10 + 1e-5
    d = weights_dirichlet(5, 1000)
    assert np.allclose(d.sum(axis=1), 10.0, rtol=1e-6) and d.min() >= 0


def test_workload_sizes():
    p, W, s = workload("prostate-2k-8plans")
    assert (p.n_pnt, p.n_dwell, W.shape) == (2000, 96, (8, 4))
    p, W, s = workload("prostate-12k-1000plans", n_plans=4)
    assert (p.n_pnt, p.n_dwell, W.shape) == (12000, 324, (4, 4))


def test_multi_patient_specs():
    specs = multi_patient_specs(64)
    assert len(specs) == 64
    for sp in specs:
        assert 12 <= sp["n_catheters"] <= 20 and 0.8 <= sp["scale"] <= 1.3
        assert 5000 <= sum(sp["n_points"]) <= 20000


def test_class_solution_patient_and_group_weights(oracle_mod):
    """The full class solution (Table 1): eight groups (surface, volume) per organ with the
    table's parameters; per-group weights w_organ N_group / N_organ make the library's
    per-group normalisation equal Eq. (obj)'s per-organ one, checked through the oracle's
    per-group objectives."""
    from synth import TABLE1, STRUCTURES, make_class_solution_patient, group_weights
    p = make_class_solution_patient(11, n_volume=(400, 80, 100, 100), n_surface=(120, 40, 60, 60))
    assert list(np.bincount(p.sid)) == [120, 400, 40, 80, 60, 100, 60, 100]
    for s, name in enumerate(STRUCTURES):
        assert tuple(p.params[2 * s]) == TABLE1[name][0] and tuple(p.params[2 * s + 1]) == TABLE1[name][1]
    rng = np.random.default_rng(0)
    w_org = rng.dirichlet(np.ones(4))
    wg = group_weights(w_org, p.sid, p.organ).astype(np.float64)
    x = rng.uniform(0.5, 1.5, p.n_dwell)
    F, _, _, f_group = oracle_mod.objective(p.A, p.sid, p.params, wg, x)
    n_group = np.bincount(p.sid).astype(np.float64)
    per_organ = sum(w_org[j] / n_group[p.organ == j].sum() * np.sum(n_group[p.organ == j] * f_group[p.organ == j])
                    for j in range(4))
    assert F == pytest.approx(per_organ, rel=1e-6)   # group weights are rounded to FP32
