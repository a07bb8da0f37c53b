"""Bounded waits of the tensor-core pipeline, made to run out on purpose (no fault).

Every mbarrier wait inside the GEMM kernels gives up after the problem's wait_limit_us.  A
limit of one microsecond is shorter than the time an accumulator takes to fill, so the
epilogue's wait for it runs out in every CTA: the kernel records the error, waits for its own
copies and MMAs in flight, frees its tensor memory and exits.  The call must return
GMCO_ECUDA promptly, and the CUDA context must stay usable: a problem with the default
limit then solves and evaluates as the oracle does, and the short-limit problem itself is
destroyed cleanly.
"""
import time

import numpy as np
import pytest

from synth import workload

pytestmark = pytest.mark.gpu


def test_wait_that_runs_out_returns_error_and_context_survives(gmco_mod, oracle_mod):
    import torch
    torch.cuda.set_device(0)
    p, W, _ = workload("prostate-12k-1000plans")
    W = W[:64]
    short = gmco_mod.Problem(p.A, p.sid, p.params, precision="bf16x2", wait_limit_us=1)
    try:
        t0 = time.perf_counter()
        with pytest.raises(gmco_mod.GmcoError) as e:
            short.solve_batch(W, max_iters=5, tol=0.0)
        elapsed = time.perf_counter() - t0
        assert e.value.status == 3   # GMCO_ECUDA
        assert "timed out" in gmco_mod.last_error()
        # the first poll sees the flag: far less than the step budget at a 1 s limit
        assert elapsed < 30.0, elapsed
        # again on the same problem: the flag was cleared and the wait runs out again
        with pytest.raises(gmco_mod.GmcoError):
            short.solve_batch(W[:8], max_iters=2, tol=0.0)
    finally:
        short.close()
    torch.cuda.synchronize()   # the context has no sticky error
    with gmco_mod.Problem(p.A, p.sid, p.params, precision="bf16x3") as ok:
        out = ok.solve_batch(W[:4], max_iters=2, tol=0.0)
    for j in range(4):
        r = oracle_mod.lbfgs(p.A, p.sid, p.params, W[j], None, max_iters=2, tol=0.0)
        assert out["iters"][j] == r["iters"] == 2
        assert abs(out["objectives"][j] / r["F"] - 1.0) <= 1e-3

