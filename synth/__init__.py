"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This package builds inputs only: voxel phase maps (microstructures) and the
stiffness tables of their phases.  It holds none of the solver's arithmetic
(no stencil, no Green operator, no FFT, no constitutive step), so it can feed
both sides without coupling them.

All random draws use ``numpy.random.Generator(PCG64(seed))``.
"""
from .microstructure import (
    centred_sphere,
    cubic_inclusion,
    laminate_x,
    random_spheres,
    voronoi_grains,
    random_rotations,
    random_phase_map,
)
from .materials import (
    isotropic_voigt,
    cubic_voigt,
    rotate_voigt,
    two_phase_table,
    polycrystal_table,
)

__all__ = [
    "centred_sphere",
    "cubic_inclusion",
    "laminate_x",
    "random_spheres",
    "voronoi_grains",
    "random_rotations",
    "random_phase_map",
    "isotropic_voigt",
    "cubic_voigt",
    "rotate_voigt",
    "two_phase_table",
    "polycrystal_table",
]
