"""Seeded synthetic SDP instances shared by the oracle, the tests and the benchmark.

This package holds input generation only: it draws problem data and builds no part of the ADMM
method. Both the CPU oracle and the CUDA path consume the arrays it returns.
"""

from .blockarrow import (  # noqa: F401
    SDPInstance,
    block_arrow_instance,
    config_instance,
    config_shapes,
    CONFIGS,
    CONIC,
    conic_extension,
    SWEEPS,
    SWEEP_MAX_ITER,
    SWEEP_TOL,
    sweep_instance,
)
