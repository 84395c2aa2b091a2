"""Seeded synthetic inputs for the spectral point-mass filter.

This package holds only input generation: the model parameters of each
workload, random stable drift matrices, true trajectories and noisy
measurements.  It contains none of the filter's arithmetic, so both the
CUDA path (through the C-ABI binding) and the FP64 oracle can take their
inputs from it without sharing any code of the method.
"""
from .configs import (  # noqa: F401
    FilterConfig, MeasModel, Scenario, ServingWorkload,
    c1_scenario, c5_serving, c6_scenario, terrain_params, c2_scenario, c3_scenario, c4_batch, small_2d_scenario,
    small_3d_scenario, random_stable_matrix, simulate,
)
