"""GB300 (sm_103a) per-pixel principal curvature from range images.

Implements the iterative quadric-patch fit of Spek, Li and Drummond, "A Fast
Method For Computing Principal Curvatures From Range Images" (arXiv
1707.00385) as hand-written CUDA kernels behind the C ABI in include/pcurv.h.
This package holds the kernels (csrc/), their build (build.py) and the
ctypes binding (pcurv.py).
"""
from .pcurv import (  # noqa: F401
    PC_OK, PC_ERR_INVALID_ARG, PC_ERR_CUDA, PC_ERR_OOM, PC_ERR_TIMEOUT, PC_ERR_UNSUPPORTED,
    Curvature, PcError, load, pc_compute, pc_compute_batch, pc_compute_batch_static, pc_compute_host, pc_compute_packed, pc_compute_packed_batch, pc_frame, pc_packed_frame,
    pc_pack_depth, pc_autotune, pc_plan_tile_height, pc_plan_lanes_per_pixel, pc_plans_export, pc_plans_import, PC_DEPTH_F16, PC_DEPTH_BF16, pc_create, pc_destroy, pc_last_error, pc_fp32_peak_kernel, pc_moments_probe,
    pc_params, pc_params_default, pc_status_string, pc_compute_host_batch, pc_backproject, pc_initial_normals,
)
