"""Plan-pool post-processing on the GPU (gmco_rtog_select, gmco_pareto_filter) against the FP64
oracle: classes, the selected index and the non-dominated flags are integers, compared exactly
(both sides take every decision in FP64 from the same FP32 DVH values)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _pool(rng, P):
    """DVH rows of a plan pool around the RTOG boundaries, with exact boundary values and ties."""
    dvh = np.empty((P, 5), np.float32)
    dvh[:, 0] = rng.choice([85.0, 89.99, 90.0, 93.0, 95.0, 97.5, 99.0], P) + rng.choice([0.0, 0.25], P)
    dvh[:, 1] = rng.uniform(95, 110, P)
    dvh[:, 2] = rng.choice([105.0, 117.5, 118.0, 121.0], P)
    dvh[:, 3] = rng.choice([0.0, 0.5, 1.0, 1.5, 2.0, 3.0], P)   # % of a 50 cc rectum: 1 cc at 2 %
    dvh[:, 4] = rng.choice([0.0, 0.5, 1.0, 2.0], P)             # % of a 100 cc bladder: 1 cc at 1 %
    return dvh


def test_rtog_select_matches_oracle(gmco_mod, oracle_mod):
    rng = np.random.default_rng(3)
    for P in (1, 7, 1000, 5000):
        dvh = _pool(rng, P)
        cls, sel = gmco_mod.rtog_select(dvh, 50.0, 100.0)
        ref_cls, ref_sel = oracle_mod.rtog_select(dvh, 50.0, 100.0)
        assert np.array_equal(cls, ref_cls) and sel == ref_sel, (P, sel, ref_sel)
    # no valid plan at all (every urethra D10 over the limit), on device buffers
    import torch
    dvh = _pool(rng, 700)
    dvh[:, 2] = 125.0
    cls, sel = gmco_mod.rtog_select(torch.from_numpy(dvh).cuda(), 50.0, 100.0)
    ref_cls, ref_sel = oracle_mod.rtog_select(dvh, 50.0, 100.0)
    assert cls.is_cuda and np.array_equal(cls.cpu().numpy(), ref_cls) and sel == ref_sel
    with pytest.raises(gmco_mod.GmcoError):
        gmco_mod.rtog_select(dvh, -1.0, 100.0)


def test_pareto_filter_matches_oracle(gmco_mod, oracle_mod):
    rng = np.random.default_rng(4)
    for P, K in ((1, 1), (6, 2), (1000, 4), (3000, 4), (513, 16)):
        obj = rng.integers(0, 12, size=(P, K)).astype(np.float64)   # many ties and duplicates
        nd = gmco_mod.pareto_filter(obj)
        assert np.array_equal(nd, oracle_mod.pareto(obj)), (P, K)
    obj = rng.uniform(0, 1, (2000, 4))
    import torch
    nd = gmco_mod.pareto_filter(torch.from_numpy(obj).cuda())
    assert nd.is_cuda and np.array_equal(nd.cpu().numpy(), oracle_mod.pareto(obj))
    with pytest.raises(gmco_mod.GmcoError):
        gmco_mod.pareto_filter(np.zeros((3, 17)))


def test_planning_flow_from_geometry(gmco_mod, oracle_mod):
    """The whole gMCO flow on the device: dose rate matrix from coordinates, a pool of plans
    solved, their DVH indices, the RTOG classes and the selected plan, and the non-dominated
    plans of the pool by (-V100, urethra D10, rectum V75, bladder V75); the classes, selection
    and flags equal the oracle's on the same DVH rows."""
    from synth import make_patient, weights_dirichlet
    p = make_patient(8, 12, 0.5, (700, 100, 150, 150))
    with gmco_mod.Problem.from_geometry(p.points, p.sid, p.dwells, p.params, precision="bf16x2") as pr:
        out = pr.solve_batch(weights_dirichlet(8, 64), max_iters=300, tol=1e-6)
    dvh = np.asarray(out["dvh"], np.float32)
    rect_cc, blad_cc = float(p.volumes_cc[2]), float(p.volumes_cc[3])
    cls, sel = gmco_mod.rtog_select(dvh, rect_cc, blad_cc)
    ref_cls, ref_sel = oracle_mod.rtog_select(dvh, rect_cc, blad_cc)
    assert np.array_equal(cls, ref_cls) and sel == ref_sel
    obj = np.column_stack([-dvh[:, 0], dvh[:, 2], dvh[:, 3], dvh[:, 4]]).astype(np.float64)
    assert np.array_equal(gmco_mod.pareto_filter(obj), oracle_mod.pareto(obj))
    assert np.all(np.isfinite(out["objectives"]))


def test_dvh_on_a_denser_point_set(gmco_mod, oracle_mod):
    """DVH indices on a separate, denser set of dose points of the same structures and dwell
    positions (Sec. 2.1, the DVH point sets): against the oracle's indices of its FP64 doses on
    that set.  V100 / V75 are point counts, so they may differ by the few points whose FP32 and
    FP64 doses fall on either side of the threshold; D90 / D10 are doses, within FP32 rounding."""
    from synth import make_patient, weights_dirichlet
    coarse = make_patient(8, 12, 0.5, (700, 100, 150, 150))
    dense = make_patient(8, 12, 0.5, (4000, 600, 900, 900))
    assert np.array_equal(coarse.dwells, dense.dwells)
    rng = np.random.default_rng(9)
    T = rng.uniform(0.5, 1.5, (6, dense.n_dwell))
    d1 = oracle_mod.dose(dense.A, np.ones(dense.n_dwell))
    T = (T * 15.0 / np.median(d1[dense.sid == 0])).astype(np.float32)   # doses around 15 Gy
    counts = np.bincount(dense.sid, minlength=4)
    with gmco_mod.Problem(dense.A, dense.sid, dense.params, precision="fp32") as pd:
        dv = pd.dvh_at(T)
        for j in range(6):
            ref = oracle_mod.dvh(oracle_mod.dose(dense.A, T[j].astype(np.float64)), dense.sid)
            assert abs(dv[j, 0] - ref[0]) <= 200.0 / counts[0] + 1e-4
            assert abs(dv[j, 3] - ref[3]) <= 200.0 / counts[2] + 1e-4
            assert abs(dv[j, 4] - ref[4]) <= 200.0 / counts[3] + 1e-4
            assert abs(dv[j, 1] / ref[1] - 1) <= 1e-5 and abs(dv[j, 2] / ref[2] - 1) <= 1e-5
        assert 0.0 < np.median(dv[:, 0]) < 100.0    # the threshold is exercised
        # plans solved on the coarse set, evaluated on the dense one (device buffers)
        with gmco_mod.Problem(coarse.A, coarse.sid, coarse.params, precision="bf16x2") as pc:
            import torch
            out = pc.solve_batch(torch.from_numpy(weights_dirichlet(8, 4)).cuda(), max_iters=200, tol=1e-6)
        dd = pd.dvh_at(out["T"])
        assert dd.is_cuda and tuple(dd.shape) == (4, 5) and bool(torch.isfinite(dd).all())
