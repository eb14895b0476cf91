"""Seeded synthetic CT-dose problems (inputs only).

This module builds the inputs of the deterministic CT dose method (meshes,
material maps, densities, multigroup cross sections, source spectra, source
positions and collimation, energy-deposition weights).  It performs none of
the method's arithmetic: no quadrature, no harmonics, no ray tracing, no
sweeps.  Both the FP64 oracle and the CUDA path consume what it returns.
"""
from .phantoms import (  # noqa: F401
    Problem,
    Source,
    tiny_cube,
    water_cylinder,
    abdomen,
    axial_scan_sources,
    extra_cylinders,
    infinite_medium_cube,
    config_problem,
    CONFIG_NAMES,
)
