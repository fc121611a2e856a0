"""Seeded synthetic single-photon lidar workloads (inputs only).

This package describes scenes -- surface depths, expected signal photons,
background rates and the instrument response -- and converts them into the
integer sampling tables that both photon samplers (the CPU oracle's and the
CUDA library's) consume.  It holds none of the reconstruction arithmetic.
"""
from .generator import (  # noqa: F401
    Irf, Scene, gaussian_irf, gamma_irf, sampling_tables, expected_histogram,
    plane_hemisphere, net_object_wall, two_layer, random_shapes, small_random, head_like,
    super_resolved, camouflage_people,
    moving_frame, make_params,
)
