"""Seeded synthetic inputs for the leaf-scattering FDTD workloads.

This package holds only input data: grid sizes, row layouts, closed-form
material indices n(lambda), kappa(lambda), CPML parameter values and seeded
label maps (the segmented cross-sections). It contains none of the FDTD
arithmetic; both the CUDA library and the FP64 oracle consume what it makes.
"""
from .configs import (  # noqa: F401
    C0, MU0, EPS0, ETA0, RunSpec, courant_dt, default_cpml,
    leaf_materials, config_c1, config_c1b, config_c2, config_c3, config_c4,
    config_c5, config_e2, crop_layout, LABELS, C2_WAVELENGTHS, POL_S, POL_P,
)
from .geometry import (  # noqa: F401
    c1_labels, c1b_labels, dicot_labels, monocot_labels, random_fields,
)
