"""Edge cases of the headline form (bf16x2) through the C ABI.

- A plan solved alone equals, bit for bit, the same plan solved inside a batch, once the
  gradient split is fixed: each plan's dose and gradient are columns of the two GEMMs that no
  other plan enters, and every reduction has a fixed order (the split plan otherwise follows
  the batch's row count).
- An empty batch is refused with GMCO_EINVAL, and the problem stays usable.
- A batch over several 128-plan tiles with a ragged last tile (300 plans: tiles of 128, 128 and
  44) reports for every plan the objective Eq. (obj) gives, in FP64, at its returned dwell
  times, within the FP32 re-evaluation's bound, including the plans of the last tile.
"""
import numpy as np
import pytest

from synth import workload

pytestmark = pytest.mark.gpu

EINVAL = 1
REPORT_TOL = 1e-5   # the FP32 re-evaluation against Eq. (obj) on the 2000-point workload


def test_single_plan_equals_its_row_in_a_batch(gmco_mod):
    p, W, _ = workload("prostate-2k-8plans")
    with gmco_mod.Problem(p.A, p.sid, p.params, precision="bf16x2", grad_split_kb=6) as pr:
        full = pr.solve_batch(W, max_iters=200, tol=1e-8)
        for j in (0, 3, 7):
            one = pr.solve_batch(W[j:j + 1], max_iters=200, tol=1e-8)
            assert np.array_equal(one["T"][0], full["T"][j]), j
            assert one["objectives"][0] == full["objectives"][j], j
            assert one["iters"][0] == full["iters"][j] and one["status"][0] == full["status"][j], j
            assert np.array_equal(one["dvh"][0], full["dvh"][j]), j


def test_empty_batch_refused(gmco_mod):
    p, W, _ = workload("prostate-2k-8plans")
    with gmco_mod.Problem(p.A, p.sid, p.params, precision="bf16x2") as pr:
        with pytest.raises(gmco_mod.GmcoError) as e:
            pr.solve_batch(W[:0], max_iters=5)
        assert e.value.status == EINVAL
        with pytest.raises(gmco_mod.GmcoError) as e:
            pr.evaluate(W[:0], np.ones((0, p.n_dwell), np.float32))
        assert e.value.status == EINVAL
        out = pr.solve_batch(W[:2], max_iters=5)   # still usable
        assert out["iters"].shape == (2,) and np.all(out["iters"] == 5)


def test_ragged_multi_tile_batch_reports_eq_obj(gmco_mod, oracle_mod):
    p, W8, _ = workload("prostate-2k-8plans")
    rng = np.random.default_rng(11)
    W = (10.0 * rng.dirichlet(np.ones(W8.shape[1]), size=300)).astype(np.float32)
    with gmco_mod.Problem(p.A, p.sid, p.params, precision="bf16x2") as pr:
        out = pr.solve_batch(W, max_iters=150, tol=0.0)
    assert out["T"].shape == (300, p.n_dwell) and np.all(out["iters"] >= 1)
    worst = 0.0
    for j in (0, 1, 127, 128, 200, 255, 256, 280, 298, 299):   # every tile, the ragged one's ends
        F_o = oracle_mod.objective(p.A, p.sid, p.params, W[j], np.sqrt(out["T"][j]))[0]
        dev = abs(out["objectives"][j] / F_o - 1.0)
        worst = max(worst, dev)
        assert dev <= REPORT_TOL, (j, out["objectives"][j], F_o)
    print(f"300 plans, worst relative deviation of the reported objective: {worst:.2e}")
