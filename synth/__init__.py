"""Seeded synthetic prostate HDR patients: the input recipe shared by tests and bench.

This package holds input generation only (geometry, dose points, dwell positions, the
point-source dose-rate matrix that the solver takes as an input, and the random hidden
weights that the multi-criteria method draws).  It holds none of the optimisation's
arithmetic: neither the oracle nor the CUDA library imports it.
"""
from .patient import (  # noqa: F401
    STRUCTURES,
    Geometry,
    WORKLOADS,
    Patient,
    make_patient,
    dwell_positions,
    dose_rate_matrix,
    class_penalty_params,
    TABLE1,
    surface_points,
    make_class_solution_patient,
    group_weights,
    weights_loguniform,
    weights_dirichlet,
    workload,
    multi_patient_specs,
    dwell_features,
    mlp_init_params,
)
