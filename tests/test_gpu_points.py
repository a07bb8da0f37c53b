"""Dose calculation points sampled on the GPU (gmco_sample_points) against the oracle's restatement
of the same rule: identical counts, ids and coordinates, bit for bit."""
import numpy as np
import pytest

from oracle import points as OP
from synth import Geometry, multi_patient_specs

pytestmark = pytest.mark.gpu


def _geo(scale):
    g = Geometry().scaled(scale)
    return {k: getattr(g, k) for k in OP.KEYS}


@pytest.mark.parametrize("scale,counts,seed", [
    (1.0, (1200, 200, 300, 300), 1),
    (0.8, (2917, 416, 833, 834), 2**63 + 11),
    (1.3, (11667, 1666, 3333, 3334), 1904015673),   # a 20000-point patient of the uneven workload
    (1.1, (0, 37, 1, 0), 5),                          # empty structures, ragged counts
])
def test_points_bit_exact(gmco_mod, scale, counts, seed):
    g = _geo(scale)
    P, sid = gmco_mod.sample_points(g, counts, seed)
    Pr, sr = OP.sample_points(g, counts, seed)
    assert np.array_equal(sid, sr)
    assert np.array_equal(P.view(np.uint32), Pr.view(np.uint32))   # every bit of every coordinate


def test_device_outputs_and_workload_patients(gmco_mod):
    import torch
    for spec in multi_patient_specs(64)[:3]:
        g = _geo(spec["scale"])
        Pd, sd = gmco_mod.sample_points(g, spec["n_points"], spec["seed"], device=True)
        assert Pd.is_cuda and sd.is_cuda
        Pr, sr = OP.sample_points(g, spec["n_points"], spec["seed"])
        assert np.array_equal(sd.cpu().numpy(), sr)
        assert np.array_equal(Pd.cpu().numpy().view(np.uint32), Pr.view(np.uint32))
    torch.cuda.synchronize()


def test_refusals(gmco_mod):
    g = _geo(1.0)
    for k, v in (("a", float("nan")), ("bladder_r", -1.0), ("urethra_r", 0.0)):
        bad = dict(g, **{k: v})
        with pytest.raises(gmco_mod.GmcoError) as e:
            gmco_mod.sample_points(bad, (10, 10, 10, 10), 1)
        assert e.value.status == gmco_mod.EINVAL
    with pytest.raises(gmco_mod.GmcoError):
        gmco_mod.sample_points(g, (0, 0, 0, 0), 1)
    # a structure covered by what it excludes runs out of candidates
    inside = dict(g, rectum_y=0.0, rectum_r=0.2, rectum_half_len=1.0)
    with pytest.raises(gmco_mod.GmcoError) as e:
        gmco_mod.sample_points(inside, (10, 10, 2000, 10), 1)
    assert e.value.status == gmco_mod.EINVAL
