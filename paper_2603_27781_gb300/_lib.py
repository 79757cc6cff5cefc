"""ctypes binding of libgs (include/gs.h): the same names, argument marshalling only.

Every computation happens in the CUDA library.  If the library has not been
built this module raises on first use; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, Structure, c_char_p, c_double, c_float, c_int, c_int32, c_int64, c_size_t, c_void_p

from . import build as _build

LIB_PATH = _build.LIB_PATH

GS_OK, GS_ERR_ARG, GS_ERR_CAPACITY, GS_ERR_CUDA, GS_ERR_TIMEOUT, GS_ERR_UNSUPPORTED, GS_ERR_CHECK = \
    0, -1, -2, -3, -4, -5, -6
GS_BWD_BLOCKS_DEFAULT, GS_BWD_BLOCKS_GROUP, GS_BWD_BLOCKS_TILE, GS_BLOCKS_QUEUE, GS_BLOCKS_RING = 0, 1, 2, 3, 4
GS_JACOBIAN_CLAMPED, GS_JACOBIAN_EXACT = 0, 1
GS_F32, GS_BF16, GS_F16 = 0, 1, 2
GS_DSR_SCRATCH_BYTES = 24832
GS_GRAD_MAP, GS_GRAD_POSE, GS_GRAD_ACCUMULATE = 1, 2, 4


class gs_camera(Structure):
    _fields_ = [("width", c_int32), ("height", c_int32), ("fx", c_float), ("fy", c_float), ("cx", c_float),
                ("cy", c_float), ("T_cw", c_float * 16)]


class gs_raster_params(Structure):
    _fields_ = [("tile", c_int32), ("alpha_min", c_float), ("alpha_max", c_float), ("T_min", c_float),
                ("z_near", c_float), ("lowpass", c_float), ("radius_sigma", c_float), ("bg_rgb", c_float * 3),
                ("fwd_px_per_thread", c_int32), ("bwd_px_per_thread", c_int32),
                ("bwd_blocks", c_int32), ("fwd_blocks", c_int32), ("jacobian", c_int32),
                ("spin_limit", c_int32), ("fwd_batch", c_int32)]


class gs_gaussians(Structure):
    _fields_ = [("n", c_int64), ("feat_dim", c_int32), ("means", c_void_p), ("quats", c_void_p),
                ("log_scales", c_void_p), ("opacity_logits", c_void_p), ("rgb", c_void_p), ("rgb_dtype", c_int32),
                ("feat", c_void_p), ("feat_dtype", c_int32)]


class gs_projected(Structure):
    _fields_ = [("uvdo", c_void_p), ("uv_lo", c_void_p), ("conic", c_void_p), ("tiles_touched", c_void_p)]


class gs_binning(Structure):
    _fields_ = [("capacity", c_int64), ("keys", c_void_p), ("vals", c_void_p), ("ranges", c_void_p),
                ("n_inst", c_void_p), ("status", c_void_p), ("tile_order", c_void_p),
                ("queue", c_void_p)]


class gs_images(Structure):
    _fields_ = [("rgb", c_void_p), ("depth", c_void_p), ("sil", c_void_p), ("feat", c_void_p),
                ("T_final", c_void_p), ("n_contrib", c_void_p), ("n_blended", c_void_p),
                ("blend_mask", c_void_p)]


class gs_splat_grads(Structure):
    _fields_ = [("uvod", c_void_p), ("conic", c_void_p), ("rgb", c_void_p)]


class gs_image_grads(Structure):
    _fields_ = [("rgb", c_void_p), ("depth", c_void_p), ("sil", c_void_p), ("feat", c_void_p),
                ("feat_coef", c_void_p), ("feat_basis", c_void_p), ("feat_rank", c_int32)]


class gs_image_grads_out(Structure):
    _fields_ = [("rgb", c_void_p), ("depth", c_void_p), ("sil", c_void_p), ("feat", c_void_p),
                ("feat_coef", c_void_p)]


class gs_field_mut(Structure):
    _fields_ = [("n", c_int64), ("feat_dim", c_int32), ("means", c_void_p), ("quats", c_void_p),
                ("log_scales", c_void_p), ("opacity_logits", c_void_p), ("rgb", c_void_p), ("feat", c_void_p)]


class gs_gaussian_grads(Structure):
    _fields_ = [("means", c_void_p), ("quats", c_void_p), ("log_scales", c_void_p), ("opacity_logits", c_void_p),
                ("rgb", c_void_p), ("feat", c_void_p)]


class gs_targets(Structure):
    _fields_ = [("rgb", c_void_p), ("depth", c_void_p), ("label", c_void_p)]


class gs_keyframes(Structure):
    _fields_ = [("capacity", c_int32), ("P", c_int64), ("rgb", c_void_p), ("depth", c_void_p), ("label", c_void_p),
                ("T_cw", c_void_p)]


class gs_loss_params(Structure):
    _fields_ = [("color", c_float), ("depth", c_float), ("sem", c_float), ("mask_mode", c_int32),
                ("tau_obs", c_float), ("n_classes", c_int32), ("ssim", c_float)]


_P = POINTER
_SIGNATURES = {
    "gs_version": (c_int, []),
    "gs_strerror": (c_char_p, [c_int]),
    "gs_cuda_error": (c_char_p, []),
    "gs_workspace_size": (c_size_t, [c_int64, c_int, _P(gs_camera), c_int64, c_int]),
    "gs_project": (c_int, [_P(gs_gaussians), _P(gs_camera), c_int, c_void_p, _P(gs_raster_params),
                           _P(gs_projected), c_void_p]),
    "gs_bin_sort": (c_int, [c_int64, _P(gs_projected), _P(gs_camera), c_int, _P(gs_raster_params), c_void_p,
                            c_size_t, _P(gs_binning), c_void_p]),
    "gs_render_fwd": (c_int, [_P(gs_gaussians), _P(gs_projected), _P(gs_binning), _P(gs_camera), c_int,
                              _P(gs_raster_params), _P(gs_images), c_void_p]),
    "gs_render_bwd": (c_int, [_P(gs_gaussians), _P(gs_projected), _P(gs_binning), _P(gs_camera), c_int,
                              _P(gs_raster_params), c_int, _P(gs_images), _P(gs_image_grads), _P(gs_splat_grads),
                              c_void_p, c_void_p]),
    "gs_splat_grads_clear": (c_int, [_P(gs_gaussians), c_int, c_int, _P(gs_splat_grads), c_void_p, c_void_p]),
    "gs_project_bwd": (c_int, [_P(gs_gaussians), _P(gs_camera), c_int, c_void_p, _P(gs_raster_params), c_int,
                               _P(gs_splat_grads), _P(gs_gaussian_grads), c_void_p, c_void_p]),
    "gs_pose_grad": (c_int, [c_int64, c_int, c_void_p, c_void_p, c_void_p]),
    "gs_loss_fwd_bwd": (c_int, [_P(gs_camera), c_int, c_int, _P(gs_images), _P(gs_targets), c_void_p, c_void_p,
                                _P(gs_loss_params), c_void_p, c_size_t, _P(gs_image_grads_out), c_void_p, c_void_p,
                                c_void_p, c_void_p, c_void_p, c_void_p]),
    "gs_loss_fwd_bwd_noalloc": (c_int, [_P(gs_camera), c_int, c_int, _P(gs_images), _P(gs_targets), c_void_p,
                                        c_void_p, _P(gs_loss_params), _P(gs_image_grads_out), c_void_p, c_void_p,
                                        c_void_p, c_void_p, c_void_p, c_void_p]),
    "gs_dsr": (c_int, [c_int64, c_void_p, c_float, c_float, c_void_p, c_size_t, c_void_p, c_void_p, c_void_p]),
    "gs_dsr_value": (c_int, [c_int64, c_void_p, c_float, c_float, c_void_p, c_void_p, c_void_p]),
    "gs_dsr_grad": (c_int, [c_int64, c_void_p, c_float, c_float, c_void_p, c_void_p, c_void_p]),
    "gs_pose_step": (c_int, [c_int, c_void_p, c_void_p, c_void_p, c_int, _P(c_double), c_double, c_double,
                             c_double, c_void_p, c_void_p]),
    "gs_adam_step": (c_int, [_P(gs_field_mut), _P(gs_gaussian_grads), c_void_p, c_int, c_void_p, _P(c_float),
                             c_double, c_double, c_double, c_void_p]),
    "gs_expand": (c_int, [_P(gs_camera), c_int, _P(gs_images), _P(gs_targets), c_float, c_void_p, c_int64,
                          _P(gs_field_mut), c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "gs_rskm_draw": (c_int, [_P(gs_keyframes), c_int32, c_int32, c_int32, c_void_p, c_int64, c_void_p, c_void_p,
                             c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
}

_lib = None


def library():
    """Loads libgs.so (raising if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgs is not built ({LIB_PATH} missing): call paper_2603_27781_gb300.build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGNATURES)


class GsError(RuntimeError):
    def __init__(self, name, status):
        msg = library().gs_strerror(status).decode()
        if status == GS_ERR_CUDA:
            msg += ": " + library().gs_cuda_error().decode()
        super().__init__(f"{name} failed: {msg} ({status})")
        self.status = status


def check(name, status):
    if status != GS_OK:
        raise GsError(name, status)
    return status


def _wrap(name):
    def call(*args):
        return getattr(library(), name)(*args)
    call.__name__ = name
    return call


gs_version = _wrap("gs_version")
gs_strerror = _wrap("gs_strerror")
gs_cuda_error = _wrap("gs_cuda_error")
gs_workspace_size = _wrap("gs_workspace_size")
gs_project = _wrap("gs_project")
gs_bin_sort = _wrap("gs_bin_sort")
gs_render_fwd = _wrap("gs_render_fwd")
gs_render_bwd = _wrap("gs_render_bwd")
gs_splat_grads_clear = _wrap("gs_splat_grads_clear")
gs_project_bwd = _wrap("gs_project_bwd")
gs_pose_grad = _wrap("gs_pose_grad")
gs_loss_fwd_bwd = _wrap("gs_loss_fwd_bwd")
gs_loss_fwd_bwd_noalloc = _wrap("gs_loss_fwd_bwd_noalloc")
gs_dsr = _wrap("gs_dsr")
gs_dsr_value = _wrap("gs_dsr_value")
gs_dsr_grad = _wrap("gs_dsr_grad")
gs_pose_step = _wrap("gs_pose_step")
gs_adam_step = _wrap("gs_adam_step")
gs_expand = _wrap("gs_expand")
gs_rskm_draw = _wrap("gs_rskm_draw")
