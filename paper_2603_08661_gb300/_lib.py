"""ctypes declarations of the libgsp C ABI (include/gsp.h), one-to-one.

Loading fails loudly: there is no CPU fallback for any entry point.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgsp.so")

c_i32, c_i64, c_f32, c_vp, c_sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_void_p, ctypes.c_size_t

GSP_OK, GSP_ERR_INVALID_ARG, GSP_ERR_CUDA, GSP_ERR_CAPACITY, GSP_ERR_TIMEOUT, GSP_ERR_WORKSPACE, \
    GSP_ERR_UNSUPPORTED = range(7)
GSP_MAX_VIEWS = 64
GSP_TILE = 16
GSP_EDGE_FUSED, GSP_EDGE_PLAIN = 0, 1
GSP_TOPK_STATIC_MAX_CAPACITY = 1 << 24
GSP_FWD_VARIANTS, GSP_BWD_VARIANTS = 6, 6


class ImageDesc(ctypes.Structure):
    _fields_ = [("rgb", c_vp), ("width", c_i32), ("height", c_i32), ("pitch_bytes", c_i64),
                ("out_offset", c_i64)]


class EdgeOpts(ctypes.Structure):
    _fields_ = [("mode", c_i32), ("use_custom_taps", c_i32), ("taps", c_f32 * 5), ("sigma", c_f32),
                ("spin_limit", c_i64), ("test_expire", c_i32), ("blocks_per_sm", c_i32)]


class Gaussians(ctypes.Structure):
    _fields_ = [("means", c_vp), ("log_scales", c_vp), ("quats", c_vp), ("opacity_logits", c_vp),
                ("sh", c_vp), ("count", c_vp), ("capacity", c_i64), ("sh_degree", c_i32)]


class Camera(ctypes.Structure):
    _fields_ = [("viewmat", c_f32 * 12), ("fx", c_f32), ("fy", c_f32), ("cx", c_f32), ("cy", c_f32),
                ("width", c_i32), ("height", c_i32), ("pixel_offset", c_i64)]


class RenderOpts(ctypes.Structure):
    _fields_ = [("pair_capacity", c_i64), ("fwd_variant", c_i32), ("bwd_variant", c_i32),
                ("pos_grad_sum", ctypes.c_void_p), ("pos_grad_count", ctypes.c_void_p),
                ("loss_pixels", c_i64), ("spin_limit", c_i64), ("test_expire", c_i32),
                ("score_event", ctypes.c_void_p), ("list_prefix", c_i64)]


class LrSchedule(ctypes.Structure):
    _fields_ = [("lr_init", c_f32 * 5), ("lr_final", c_f32 * 5), ("steps", c_i32)]


class SelectOpts(ctypes.Structure):
    _fields_ = [("pos_grad_sum", c_vp), ("pos_grad_count", c_vp), ("threshold", c_f32), ("exp_variates", c_vp),
                ("budget", c_i64), ("spin_limit", c_i64), ("test_expire", c_i32)]


class LasParams(ctypes.Structure):
    _fields_ = [("k_off", c_f32), ("long_factor", c_f32), ("other_factor", c_f32), ("beta", c_f32)]


P = ctypes.POINTER

# name -> (restype, argtypes), exactly the declarations of include/gsp.h
SIGNATURES = {
    "gsp_status_string": (ctypes.c_char_p, [c_i32]),
    "gsp_last_cuda_error": (c_i32, []),
    "gsp_version": (c_i32, []),
    "gsp_kernel_launch_count": (c_i64, []),
    "gsp_stage_timer_arm": (c_i32, [ctypes.c_char_p, c_i32]),
    "gsp_stage_timer_read": (c_i32, [P(c_f32), P(c_i32)]),
    "gsp_edge_opts_default": (None, [P(EdgeOpts)]),
    "gsp_edge_map_workspace_size": (c_sz, [P(ImageDesc), c_i32, P(EdgeOpts)]),
    "gsp_edge_map": (c_i32, [P(ImageDesc), c_i32, c_vp, c_vp, c_vp, P(EdgeOpts), c_vp, c_sz, c_vp, c_vp]),
    "gsp_render_workspace_size": (c_sz, [c_i64, c_i32, P(Camera), c_i32, P(RenderOpts)]),
    "gsp_render_fwd": (c_i32, [P(Gaussians), P(Camera), c_i32, P(ImageDesc), c_vp, c_vp, c_vp, c_vp, c_vp,
                               c_vp, P(RenderOpts), c_vp, c_sz, c_vp, c_vp]),
    "gsp_render_pair_count_ptr": (c_vp, [c_vp, c_i64, c_i32, P(Camera), c_i32, P(RenderOpts)]),
    "gsp_render_bwd": (c_i32, [P(Gaussians), P(Camera), c_i32, P(ImageDesc), c_vp, c_vp, c_vp, c_vp, c_vp,
                               c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_i32, P(RenderOpts), c_vp, c_sz, c_vp,
                               c_vp]),
    "gsp_las_params_paper": (None, [P(LasParams)]),
    "gsp_las_workspace_size": (c_sz, [c_i64]),
    "gsp_topk_mask": (c_i32, [c_vp, c_vp, c_i64, c_i64, c_vp, c_vp, c_vp, c_sz, c_vp, c_vp]),
    "gsp_topk_mask_gated": (c_i32, [c_vp, c_vp, c_vp, c_f32, c_vp, c_i64, c_i64, c_vp, c_vp, c_vp, c_sz, c_vp, c_vp]),
    "gsp_sample_mask": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_i64, c_vp, c_vp, c_vp, c_sz, c_vp, c_vp]),
    "gsp_select_mask": (c_i32, [c_vp, c_vp, c_i64, c_i64, P(SelectOpts), c_vp, c_vp, c_vp, c_sz, c_vp, c_vp]),
    "gsp_las_split": (c_i32, [P(Gaussians), c_vp, c_vp, c_i64, P(LasParams), c_vp, c_sz, c_vp, c_vp]),
    "gsp_topk_mask_static": (c_i32, [c_vp, c_vp, c_i64, c_i64, c_vp, c_vp, c_vp, c_vp]),
    "gsp_sgd_step": (c_i32, [P(Gaussians), c_vp, c_vp, c_vp, c_vp, c_vp, c_f32, c_vp]),
    "gsp_sgd_step_scheduled": (c_i32, [P(Gaussians), c_vp, c_vp, c_vp, c_vp, c_vp, P(LrSchedule), c_vp, c_vp]),
}

_lib = None


def load(path: str | None = None):
    """Load libgsp.so (or the build GSP_LIBRARY names, e.g. the bounds-checked
    libgsp_debug.so) and declare every entry point; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = os.environ.get("GSP_LIBRARY") or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"libgsp.so not built at {path}; run `python paper_2603_08661_gb300/build.py`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class GspError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        msg = lib.gsp_status_string(status).decode()
        if status == GSP_ERR_CUDA:
            msg += f" (cudaError {lib.gsp_last_cuda_error()})"
        super().__init__(f"{where}: {msg}")
        self.status = status


def check(status: int, where: str):
    if status != GSP_OK:
        raise GspError(status, where)
