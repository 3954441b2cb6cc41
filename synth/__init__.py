"""Seeded synthetic seismic gathers shared by the tests, the benchmark and the smoke check.

This package holds input generation only (wavelets, event traveltimes, noise).  It
contains none of the misfit's arithmetic, so both the FP64 oracle and the CUDA path
can be fed from it without sharing any part of the method.
"""

from .gathers import (  # noqa: F401
    ricker,
    gather_pair_hyperbolic,
    shift_sweep_1d,
    gather_pair_transmissive,
    batch_uneven_hyperbolic,
    gather_pair_reflective,
    gather_pair_marine,
    marine_shot,
    workload,
)
