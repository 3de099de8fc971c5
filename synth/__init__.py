"""Seeded synthetic interferogram stacks shaped like the paper's workload.

This module is the only code shared by the FP64 oracle side and the CUDA side.  It
holds a forward model of the recording (object field + tilted local oscillator ->
camera counts), never a step of the reconstruction (no rescaling, no Fresnel
transform, no sweep-axis transform).
"""

from .interferograms import (  # noqa: F401
    OPTICS,
    Scatterer,
    Workload,
    sweep_wavelengths,
    point_scatterer_stack,
    speckle_stack,
    workload,
    WORKLOADS,
)
