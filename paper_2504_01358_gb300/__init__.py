"""GB300-native screen-space global illumination (arXiv 2504.01358's hot path).

The compute lives in libssgi.so (CUDA, sm_103a, C ABI in include/ssgi.h); this package is
the thin binding: ssgi.py mirrors the C entry points for torch CUDA tensors, and serve.py
drives the serving loop.
"""
from .ssgi import (ssgi_tonemap_srgb, ssgi_l2_loss_srgb, ssgi_env_keyframe_lerp, ssgi_env_keyframe_lerp_backward, ssgi_keyframe_of, EnvMap, FramePipeline, GBuffer, SSGIFunction, TraceParams, cameras, params_of, ssgi_backward,
                   ssgi_backward_noalloc, ssgi_backward_workspace_bytes, ssgi_build_brdf_lut, ssgi_build_env_mips, ssgi_build_hiz, ssgi_build_hiz_normals, ssgi_composite_gbuffer, ssgi_depth_normals,
                   ssgi_env_levels, ssgi_env_mip_floats, ssgi_hiz_floats, ssgi_l2_loss, ssgi_read_bandwidth_probe, ssgi_render,
                   ssgi_shade_direct, ssgi_status_string, ssgi_step_fused,
                   ssgi_step_fused_check, ssgi_step_fused_phase_ns, ssgi_step_fused_set_wait_limit, ssgi_step_fused_workspace_bytes, ssgi_trace_indirect, ssgi_version, to_device_workload)

__all__ = [
    "ssgi_tonemap_srgb", "ssgi_l2_loss_srgb", "ssgi_env_keyframe_lerp", "ssgi_env_keyframe_lerp_backward", "ssgi_keyframe_of",
    "EnvMap", "FramePipeline", "GBuffer", "SSGIFunction", "TraceParams", "cameras", "params_of", "ssgi_backward",
    "ssgi_backward_noalloc", "ssgi_backward_workspace_bytes", "ssgi_build_brdf_lut", "ssgi_build_env_mips", "ssgi_build_hiz", "ssgi_build_hiz_normals", "ssgi_composite_gbuffer", "ssgi_depth_normals",
    "ssgi_env_levels", "ssgi_env_mip_floats", "ssgi_hiz_floats", "ssgi_l2_loss", "ssgi_read_bandwidth_probe", "ssgi_render",
    "ssgi_shade_direct", "ssgi_status_string", "ssgi_step_fused",
    "ssgi_step_fused_check", "ssgi_step_fused_phase_ns", "ssgi_step_fused_set_wait_limit", "ssgi_step_fused_workspace_bytes", "ssgi_trace_indirect", "ssgi_version", "to_device_workload",
]
