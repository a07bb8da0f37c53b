"""B300-native batched gL-BFGS Pareto-plan optimiser (arXiv 1904.01567, gMCO).

The compute path is the CUDA library libgmco.so (paper_1904_01567_b300/csrc, C ABI in
include/gmco.h); this package only marshals arguments to it.
"""
from .gmco import (  # noqa: F401
    Problem,
    Multi,
    Mlp,
    warm_start,
    MLP_NPARAM,
    MLP_NFEAT,
    OK,
    EINVAL,
    ENOMEM,
    ECUDA,
    ETIMEOUT,
    EUNSUPPORTED,
    GmcoError,
    create_problem,
    default_source,
    dose_rate_matrix,
    destroy_problem,
    solve_batch,
    evaluate,
    evaluate_noalloc,
    dvh_from_dose,
    profile_evaluate,
    problem_info,
    last_launch_count,
    status_string,
    default_options,
    load,
    LIB_PATH,
    PREC,
    PLAN_STATUS,
    DVH_K,
    DVH_NAMES,
)
