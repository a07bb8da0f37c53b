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
        Xs = [np.random.default_rng(seed).uniform(0.3, 1.7, (8, p.n_dwell)).astype(np.float32)
              for seed in (0, 1)]
        refs = [pr.evaluate(W, X, objectives=True, grad=True) for X in Xs]
        Xd = [torch.from_numpy(X).cuda() for X in Xs]
        # outputs allocated up front, as a caller that cannot allocate would hold them
        F_out = torch.empty(8, dtype=torch.float64, device="cuda")
        g_out = torch.empty((8, p.n_dwell), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        for X, ref in zip(Xd, refs):
            pr.evaluate_noalloc(Wd, X, objectives=F_out, grad=g_out)
            torch.cuda.synchronize()
            F = F_out.cpu().numpy()
            g = g_out.cpu().numpy()
            assert np.all(np.abs(F / ref["objectives"] - 1.0) <= 1e-5)
            for j in range(8):
                assert np.max(np.abs(g[j] - ref["grad"][j])) <= 1e-5 * np.max(np.abs(ref["grad"][j]))
        # after those calls (the first one on this device resolved the scratch array's
        # address), a further call changes neither torch's allocations nor the device's free
        # memory: the call allocates nothing
        alloc0 = torch.cuda.memory_allocated()
        free0 = torch.cuda.mem_get_info()[0]
        pr.evaluate_noalloc(Wd, Xd[0], objectives=F_out, grad=g_out)
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == alloc0
        assert torch.cuda.mem_get_info()[0] == free0
        assert np.all(np.abs(F_out.cpu().numpy() / refs[0]["objectives"] - 1.0) <= 1e-5)


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
        # shapes that do not match the problem are refused before the C call
        with pytest.raises(ValueError):
            pr.evaluate_noalloc(big[:8], X[:8, :-1])
        with pytest.raises(ValueError):
            pr.evaluate_noalloc(big[:8, :3], X[:8])
        # host buffers are refused: staging them would need device scratch
        Xh = np.ones((8, p.n_dwell), np.float32)
        Fh = np.zeros(8)
        rc = gmco_mod.load().gmco_evaluate_noalloc(pr.handle, W.ctypes.data, 8, Xh.ctypes.data,
                                                   Fh.ctypes.data, None, None)
        assert rc == 1   # GMCO_EINVAL
