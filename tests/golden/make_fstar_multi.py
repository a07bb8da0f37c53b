"""Writes tests/golden/fstar_multi64_sample.txt: the exact FP64 optimum F* of a seeded sample
of plans of the 64-patient workload (uneven patients, 256 Dirichlet plans each).

Calls only the oracle package and the seeded input generator: a 300-iteration oracle L-BFGS
run gives a warm start, then oracle.fstar computes the exact minimum of Eq. (obj) over t >= 0
and certifies it by the KKT conditions (as tests/golden/make_fstar.py does for one patient).

usage: python tests/golden/make_fstar_multi.py [plans_per_patient] [n_workers]
"""
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

N_PATIENTS, PLANS = 64, 256
SAMPLE_SEED = 19040157
_CTX = {}


def sample_plans(n_per_patient):
    """(patient, plan) pairs of the sample, n_per_patient seeded plans of each patient."""
    rng = np.random.default_rng(SAMPLE_SEED)
    return [(p, int(j)) for p in range(N_PATIENTS)
            for j in np.sort(rng.choice(PLANS, n_per_patient, replace=False))]


def _solve(task):
    import oracle
    from synth import make_patient, multi_patient_specs, weights_dirichlet
    p, j = task
    key = p
    if _CTX.get("key") != key:
        s = multi_patient_specs(N_PATIENTS)[p]
        _CTX.update(key=key, pat=make_patient(s["seed"], s["n_catheters"], s["dwell_step"],
                                              s["n_points"], s["scale"]),
                    W=weights_dirichlet(s["seed"], PLANS))
    pat, W = _CTX["pat"], _CTX["W"]
    warm = oracle.lbfgs(pat.A, pat.sid, pat.params, W[j], max_iters=300, tol=0.0)
    r = oracle.fstar(pat.A, pat.sid, pat.params, W[j], t_init=warm["t"])
    return p, j, r["F"], r["kkt"], r["rounds"]


def main():
    n_per = int(sys.argv[1]) if len(sys.argv) > 1 else 4
    nw = int(sys.argv[2]) if len(sys.argv) > 2 else max(1, (os.cpu_count() or 2) - 1)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    import oracle
    oracle.build()
    tasks = sample_plans(n_per)
    t0 = time.time()
    rows = {}
    with mp.get_context("spawn").Pool(nw) as pool:
        # consecutive tasks of one patient go to one worker, which keeps the patient cached
        for p, j, F, kkt, rounds in pool.imap_unordered(_solve, tasks, chunksize=n_per):
            rows[(p, j)] = (F, kkt, rounds)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fstar_multi64_sample.txt")
    with open(out, "w") as f:
        f.write(f"# exact FP64 optimum F* of {n_per} seeded plans (seed {SAMPLE_SEED}) of each of the "
                f"{N_PATIENTS} patients of the uneven-batching workload ({PLANS} plans each)\n")
        f.write("# written by tests/golden/make_fstar_multi.py (oracle.lbfgs warm start + "
                "oracle.fstar active-set NNLS, KKT-certified)\n")
        f.write("# patient plan F_star kkt_residual rounds\n")
        for p, j in tasks:
            F, kkt, rounds = rows[(p, j)]
            f.write(f"{p} {j} {F:.17g} {kkt:.3e} {rounds}\n")
    print(f"wrote {out} ({len(tasks)} plans, {time.time() - t0:.1f} s, max kkt "
          f"{max(v[1] for v in rows.values()):.2e})")


if __name__ == "__main__":
    main()
