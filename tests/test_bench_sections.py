"""Host logic of the benchmark's annealing and stopping-criterion sections, run on the CPU with
stand-ins for the library and the CUDA events (no device): the keys of their JSON objects, the
ratios they derive and the per-structure one-hot weights they evaluate with; and the reference
arm's line (the oracle on host cores), which states the GPU arm's workload config."""
import sys
import types
import os

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


class _Event:
    def __init__(self, enable_timing=True):
        pass

    def record(self, stream=None):
        pass

    def elapsed_time(self, other):
        return 2.0


_fake_torch = types.SimpleNamespace(
    cuda=types.SimpleNamespace(Event=_Event, synchronize=lambda: None),
    sqrt=torch.sqrt, zeros=lambda shape, dtype, device: torch.zeros(shape, dtype=dtype),
    float32=torch.float32)


class _Solver:
    def __init__(self):
        self.tols = []

    def solve_batch(self, W, max_iters, tol, stream=None, allow_timeout=False):
        self.tols.append(tol)
        P = W.shape[0]
        return {"T": torch.full((P, 3), 4.0), "iters": torch.full((P,), 9, dtype=torch.int32),
                "objectives": torch.full((P,), 2.0, dtype=torch.float64)}

    def solve_sa(self, W, iterations, stream=None):
        P = W.shape[0]
        return {"objectives": torch.full((P,), 3.0, dtype=torch.float64),
                "accepts": torch.full((P,), iterations // 2, dtype=torch.int32)}

    def last_launch_count(self):
        return 5


def test_eps_sweep_section_host_logic():
    seen = []

    class _P32:
        def __init__(self, *a, **k):
            pass

        def __enter__(self):
            return self

        def __exit__(self, *a):
            return False

        def evaluate(self, Wk, X, objectives, grad):
            seen.append(Wk.clone())
            return {"objectives": torch.arange(X.shape[0], dtype=torch.float64)}

    g = types.SimpleNamespace(Problem=_P32, pareto_filter=lambda f: (np.arange(len(f)) < 2).astype(np.int32))
    pat = types.SimpleNamespace(A=None, sid=None, params=np.zeros((4, 4)))
    solver = _Solver()
    fstar = np.array([2.0, 2.0, 1.0, 2.0, 2.0])
    r = bench.eps_sweep_section(g, _fake_torch, solver, pat, torch.zeros(5, 4), 10, None, fstar,
                                eps_list=(1e-7, 1e-3), fobj=lambda out: out["objectives"].cpu().numpy())
    assert [row["eps"] for row in r["rows"]] == [1e-7, 1e-3]
    assert solver.tols == [1e-7, 1e-7, 1e-3, 1e-3]           # one warm-up and one timed solve each
    assert all(row["frac_nondominated"] == 0.4 and row["speedup_vs_first"] == 1.0 for row in r["rows"])
    assert len(seen) == 8                                    # one evaluation per structure and eps
    assert all(row["median_gap_vs_fstar"] == 0.0 and row["plans_within_1e-4"] == 4 for row in r["rows"])
    for k, Wk in enumerate(seen[:4]):
        assert torch.equal(Wk, torch.nn.functional.one_hot(torch.full((5,), k), 4).float())


def test_gsa_section_host_logic():
    fstar = np.full(4, 1.5)
    r = bench.gsa_section(None, _fake_torch, _Solver(), torch.zeros(4, 4), fstar, 100, 8.0, None)
    assert r["iterations"] == 100 and r["plans"] == 4 and r["ms"] == 2.0
    assert r["plan_iterations_per_s"] == 4 * 100 / 2e-3
    assert r["rel_gap_vs_fstar"]["median"] == 1.0 and r["plans_within_1e-4"] == 0
    assert r["accept_rate_median"] == 0.5 and r["ms_ratio_gsa_over_lbfgs"] == 0.25


def test_section_summary_keeps_key_figures():
    sec = {"rows": [{"eps": 1e-3, "ms": 12.3456, "frac_nondominated": 0.56789, "median_gap_vs_fstar": 1e-3}]}
    assert bench.section_summary("eps_sweep", sec) == {"0.001": [12.35, 0.5679, 1e-3]}
    assert bench.section_summary("gsa", {"error": "boom"}) == {"error": "boom"}
    assert "summary_error" in bench.section_summary("gsa", {"ms": 1.0})
    d = {"stop_rule_1e-4": {"ms": 12.34, "iters_median": 700.0, "within_1e-4": 5},
         "iters_to_1e-4": {"median": 800.0}, "budgets": {"800": {"ms": 3.21, "within_1e-4": 4}}}
    assert bench.section_summary("warm_start", {"by_start": {"bf16x2_warm": d}}) == {
        "bf16x2_warm": {"stop_1e-4": [12.3, 700.0, 5], "iters_to_1e-4": 800.0, "800": [3.2, 4]}}


def test_reference_arm_states_the_gpu_arms_config():
    """The reference arm (the FP64 oracle on host cores, timed on a bounded sample) prints the
    same workload config as the GPU arm would for the same arguments, and describes its sample
    in cpu_baseline.sample."""
    import json
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          "--workload", "prostate-2k-8plans", "--steps", "1", "--warmup", "0",
                          "--cpu-sample", "2"],
                         capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    from synth import workload
    pat, W, _ = workload("prostate-2k-8plans")
    saved = sys.argv
    try:
        sys.argv = ["bench.py", "--workload", "prostate-2k-8plans"]
        args = bench.parse_args()
    finally:
        sys.argv = saved
    want = dict(bench.workload_config(args, pat, W.shape[0]), parallelism="replicas1")
    assert line["config"] == want
    assert line["data"] == bench.DATA
    assert line["impl"] == "reference" and line["cpu_baseline"]["kind"] == "oracle"
    assert "first 2 plans" in line["cpu_baseline"]["sample"]
