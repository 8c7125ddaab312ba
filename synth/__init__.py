"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This package holds no arithmetic of the method: it only draws media (refractive
index maps without absorbing layers) and sources from seeded generators.
"""
from .media import (  # noqa: F401
    frequency_batch,
    spheres_medium,
    fill_spheres_medium,
    gaussian_random_field_medium,
    point_source,
    gaussian_beam_plane_source,
    packed_spheres_medium,
    plane_source,
    random_field,
    CONFIGS,
    config_problem,
)
