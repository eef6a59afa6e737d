"""Seeded synthetic inputs shared by the FP64 oracle and the GPU path.

This package holds only input generation: workload descriptions (grid sizes,
level strides, medium family, contrast, seed) and the high-contrast media
(kappa per element and continuum label per element) sampled on a macropoint's
RVE grid. It contains none of the homogenization arithmetic (no stiffness,
constraints, solves or effective coefficients), so that the oracle and the
CUDA path can both consume its output without sharing method code.
"""
from .configs import Workload, WORKLOADS, workload, small_workload
from .media import media, macro_points_xyz, counter_uniform

__all__ = ["Workload", "WORKLOADS", "workload", "small_workload", "media",
           "macro_points_xyz", "counter_uniform"]
