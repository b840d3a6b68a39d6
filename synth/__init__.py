"""Seeded synthetic workloads for the TaCo query path.

This package only draws random inputs (data points, queries, parameters). It holds
none of the method's arithmetic, so both the FP64 oracle and the GPU library may use
it without sharing any step of the computation.
"""
from .workloads import (  # noqa: F401
    WORKLOADS,
    Workload,
    make_workload,
    gmm_isotropic,
    gmm_integer,
    powerlaw_mixture,
    gmm_unit_normalised,
    gmm_anisotropic,
    budget_from_alpha,
    target_from_beta,
)
