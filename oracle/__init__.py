"""FP64 CPU oracle (test infrastructure only).

Only the test-suite, the smoke check and the benchmark's CPU-baseline / reference leg use
this package.  The product path (paper_1904_01567_b300) never imports it.
"""
from .oracle import (  # noqa: F401
    build,
    load,
    dose,
    dose_rate,
    DEFAULT_SOURCE,
    rtog_select,
    pareto,
    RTOG,
    point_penalty,
    point_dpenalty,
    objective,
    two_loop,
    lbfgs,
    lbfgs_batch,
    splitmix64,
    sa,
    sa_batch,
    dvh,
    CONVERGED,
    MAXITER,
    LSFAIL,
    NONFINITE,
)
from .optimum import fstar, objective_t, kkt_residual  # noqa: F401,E402
from . import mlp  # noqa: F401,E402
from . import points  # noqa: F401,E402
