"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This package holds geometry and random-number generation only (dielectric
inclusions sampled on the Yee grid, smoothed random fields, Bloch k-point
paths, random test vectors).  It contains none of the eigensolver's
arithmetic: both the oracle and the CUDA library consume the arrays produced
here, each with its own implementation of the method.
"""

from .media import (  # noqa: F401
    Medium,
    biisotropic_sphere,
    bz_path_midpoints,
    chiral_sphere,
    homogeneous,
    pseudochiral_cylinders,
    random_complex,
    smoothed_chiral_field,
    workload,
    WORKLOADS,
)
