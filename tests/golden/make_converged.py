"""Writes tests/golden/converged_<workload>.txt: what the FP64 oracle reaches on a plan sample.

For each sampled plan of the workload, under the benchmark's stopping rule (relative objective
change tol = 1e-10, at most 3000 accepted iterations and 3000 objective evaluations per plan):

  - the oracle's own L-BFGS (oracle.lbfgs, FP64, Sec. 2.2.2-2.2.3): final F, iterations, status,
    and V100 / D90 (Sec. 2.3.1) of its final doses;
  - the exact optimum (oracle.fstar, KKT-certified, started from that L-BFGS point): F* and
    V100 / D90 of its doses.

The GPU tests grade the GPU's converged plans against these: how many land within 1e-4 of F*
(against how many the oracle lands there under the same rule), and how many have V100 and D90
within 0.5 percentage points of the optimum's (against the oracle's own count).

Calls only the oracle package and the seeded input generator.

usage: python tests/golden/make_converged.py <workload> [n_sample] [n_workers]
       (n_sample 0 = every plan; otherwise a seeded sample of that many plan indices)
"""
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

TOL, MAX_ITERS, MAX_EVALS = 1e-10, 3000, 3000
SAMPLE_SEED = 19040156
_CTX = {}


def sample_indices(P, n):
    """The plan indices of the sample: every plan for n = 0 or n >= P, else n seeded ones."""
    if n <= 0 or n >= P:
        return np.arange(P)
    return np.sort(np.random.default_rng(SAMPLE_SEED).choice(P, n, replace=False))


def _init(name):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from synth import workload
    pat, W, _ = workload(name)
    _CTX.update(pat=pat, W=W)


def _solve(j):
    import oracle
    pat, W = _CTX["pat"], _CTX["W"]
    r = oracle.lbfgs(pat.A, pat.sid, pat.params, W[j], max_iters=MAX_ITERS, tol=TOL,
                     max_evals=MAX_EVALS)
    dvh_l = oracle.dvh(oracle.dose(pat.A, r["t"]), pat.sid, 4, 15.0)
    s = oracle.fstar(pat.A, pat.sid, pat.params, W[j], t_init=r["t"])
    dvh_s = oracle.dvh(oracle.dose(pat.A, s["t"]), pat.sid, 4, 15.0)
    return (j, r["F"], r["iters"], r["status"], dvh_l[0], dvh_l[1], s["F"], dvh_s[0], dvh_s[1],
            s["kkt"])


def main():
    name = sys.argv[1]
    n_sample = int(sys.argv[2]) if len(sys.argv) > 2 else 0
    nw = int(sys.argv[3]) if len(sys.argv) > 3 else max(1, (os.cpu_count() or 2) - 1)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    import oracle
    oracle.build()
    from synth import workload
    _, W, _ = workload(name)
    idx = sample_indices(W.shape[0], n_sample)
    t0 = time.time()
    rows = {}
    with mp.get_context("spawn").Pool(nw, initializer=_init, initargs=(name,)) as pool:
        for row in pool.imap_unordered(_solve, [int(j) for j in idx]):
            rows[row[0]] = row
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"converged_{name}.txt")
    with open(out, "w") as f:
        f.write(f"# FP64 oracle on workload {name}, plan sample seed {SAMPLE_SEED} "
                f"({len(idx)} plans; 0 = all)\n")
        f.write(f"# rule: tol {TOL:g}, max_iters {MAX_ITERS}, max_evals {MAX_EVALS}\n")
        f.write("# written by tests/golden/make_converged.py (oracle.lbfgs, oracle.fstar, "
                "oracle.dvh)\n")
        f.write("# plan F_lbfgs iters status V100_lbfgs D90_lbfgs F_star V100_star D90_star "
                "kkt\n")
        for j in idx:
            r = rows[int(j)]
            f.write(f"{r[0]} {r[1]:.17g} {r[2]} {r[3]} {r[4]:.6f} {r[5]:.6f} {r[6]:.17g} "
                    f"{r[7]:.6f} {r[8]:.6f} {r[9]:.3e}\n")
    print(f"wrote {out} ({len(idx)} plans, {time.time() - t0:.1f} s)")


if __name__ == "__main__":
    main()
