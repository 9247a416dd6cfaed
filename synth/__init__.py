"""Seeded synthetic inputs for occlusion-point reuse.

This package only builds input data: triangle soups, cameras, area lights,
receiver grids and neighbour-offset tables.  It holds none of the method's
arithmetic (no ray tracing, sampling, densities or MIS), so both the CUDA
library and the FP64 CPU oracle can consume its outputs without sharing code.
"""
from .scenes import (  # noqa: F401
    Camera,
    RectLight,
    Scene,
    camera_c1,
    camera_c2,
    disk_offsets,
    light_c3,
    receiver_grid,
    scene_c1,
    scene_fully_blocked,
    scene_half_plane,
    scene_parallel_plane,
    scene_plane_only,
    scene_terrain,
    serving_views,
)
