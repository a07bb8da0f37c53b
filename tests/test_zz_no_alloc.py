"""The allocation-free evaluation entry point (gmco_evaluate_noalloc) through the C ABI.

Callers that cannot allocate device memory while they run use this call; its scratch is a
fixed array inside the library.  It must agree with gmco_evaluate (the allocating path) on two
calls in a row, since the second call reuses the array the first one left behind.
"""
import numpy as np
import pytest

from synth import workload

pytestmark = pytest.mark.gpu


def test_noalloc_matches_evaluate_twice(gmco_mod):
    import torch
    torch.cuda.set_device(0)
    p, W, _ = workload("prostate-2k-8plans")
    with gmco_mod.Problem(p.A, p.sid, p.params, precision="fp32") as pr:
        Wd = torch.from_numpy(W).cuda()
        for seed in (0, 1):
            X = np.random.default_rng(seed).uniform(0.3, 1.7, (8, p.n_dwell)).astype(np.float32)
            ref = pr.evaluate(W, X, objectives=True, grad=True)
            out = pr.evaluate_noalloc(Wd, torch.from_numpy(X).cuda())
            torch.cuda.synchronize()
            F = out["objectives"].cpu().numpy()
            g = out["grad"].cpu().numpy()
            assert np.all(np.abs(F / ref["objectives"] - 1.0) <= 1e-5)
            for j in range(8):
                assert np.max(np.abs(g[j] - ref["grad"][j])) <= 1e-5 * np.max(np.abs(ref["grad"][j]))


def test_noalloc_rejects_oversized_and_host_buffers(gmco_mod):
    import torch
    torch.cuda.set_device(0)
    p, W, _ = workload("prostate-2k-8plans")
    with gmco_mod.Problem(p.A, p.sid, p.params, precision="fp32") as pr:
        big = torch.ones((2000, 4), dtype=torch.float32, device="cuda")
        X = torch.ones((2000, p.n_dwell), dtype=torch.float32, device="cuda")
        with pytest.raises(gmco_mod.GmcoError) as e:
            pr.evaluate_noalloc(big, X)
        assert e.value.status == 5   # GMCO_EUNSUPPORTED: beyond the fixed scratch array
        # host buffers are refused: staging them would need device scratch
        Xh = np.ones((8, p.n_dwell), np.float32)
        Fh = np.zeros(8)
        rc = gmco_mod.load().gmco_evaluate_noalloc(pr.handle, W.ctypes.data, 8, Xh.ctypes.data,
                                                   Fh.ctypes.data, None, None)
        assert rc == 1   # GMCO_EINVAL
