"""Writes tests/golden/fstar_<workload>.txt: the exact FP64 optimum F* of every plan.

Calls only the oracle package (and the seeded input generator): a 300-iteration oracle
L-BFGS run gives a warm start, then oracle.optimum.fstar computes the exact minimum of
Eq. (obj) over t >= 0 and certifies it by the KKT conditions.

usage: python tests/golden/make_fstar.py <workload> [n_workers]
"""
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

_CTX = {}


def _init(name):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from synth import workload
    pat, W, _ = workload(name)
    _CTX.update(pat=pat, W=W)


def _solve(j):
    import oracle
    pat, W = _CTX["pat"], _CTX["W"]
    warm = oracle.lbfgs(pat.A, pat.sid, pat.params, W[j], max_iters=300, tol=0.0)
    r = oracle.fstar(pat.A, pat.sid, pat.params, W[j], t_init=warm["t"])
    return j, r["F"], r["kkt"], r["rounds"]


def main():
    name = sys.argv[1]
    nw = int(sys.argv[2]) if len(sys.argv) > 2 else max(1, (os.cpu_count() or 2) - 1)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    import oracle
    oracle.build()
    from synth import workload
    _, W, _ = workload(name)
    P = W.shape[0]
    t0 = time.time()
    rows = [None] * P
    with mp.get_context("spawn").Pool(nw, initializer=_init, initargs=(name,)) as pool:
        for j, F, kkt, rounds in pool.imap_unordered(_solve, range(P)):
            rows[j] = (j, F, kkt, rounds)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"fstar_{name}.txt")
    with open(out, "w") as f:
        f.write(f"# exact FP64 optimum F* = min_(t>=0) F(t) per plan of workload {name}\n")
        f.write("# written by tests/golden/make_fstar.py (oracle.lbfgs warm start + "
                "oracle.fstar active-set NNLS, KKT-certified)\n")
        f.write("# plan F_star kkt_residual rounds\n")
        for j, F, kkt, rounds in rows:
            f.write(f"{j} {F:.17g} {kkt:.3e} {rounds}\n")
    print(f"wrote {out} ({P} plans, {time.time() - t0:.1f} s, max kkt "
          f"{max(r[2] for r in rows):.2e})")


if __name__ == "__main__":
    main()
