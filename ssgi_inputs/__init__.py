"""Seeded synthetic inputs (scenes, cameras, env maps, targets) shared by the oracle and the library."""
from .scenes import (CAM_FLOATS, TraceParams, Workload, config1, config2, config3, config4, look_at,
                     lognormal_env, make_scene, pixel_rays, raycast_gbuffer, single_view, small_case,
                     uniform_target, Scene, Box, Quad, Material)

__all__ = [
    "CAM_FLOATS", "TraceParams", "Workload", "config1", "config2", "config3", "config4", "look_at",
    "lognormal_env", "make_scene", "pixel_rays", "raycast_gbuffer", "single_view", "small_case",
    "uniform_target", "Scene", "Box", "Quad", "Material",
]
