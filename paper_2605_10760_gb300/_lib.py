"""ctypes declarations of the libgs C ABI (include/gs.h).  Argument marshalling only.

Loading fails loudly: if libgs.so cannot be built or loaded there is no other implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import re

_HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(_HERE), "include", "gs.h")

GS_OK = 0
GS_ERR_INVALID_ARG = -1
GS_ERR_CAPACITY = -2
GS_ERR_TIMEOUT = -3
GS_ERR_CUDA = -4
GS_ERR_DEVICE_FAULT = -5
GS_ERR_TOO_LARGE = -6
GS_SORT_TILE_BUCKET = 0
GS_SORT_ONESWEEP = 1
GS_SSIM_NOALLOC_MAX_PLANE = 1 << 20
GS_MAX_VIEWS = 1024


class GsError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (what, error_string(code), code))


class gs_camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float)]


class gs_params(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("near_plane", C.c_float), ("dilation", C.c_float),
                ("radius_sigmas", C.c_float), ("alpha_max", C.c_float), ("alpha_min", C.c_float),
                ("t_min", C.c_float), ("bg", C.c_float * 3), ("sort_mode", C.c_int32),
                ("batch_records", C.c_int32)]


class gs_problem(C.Structure):
    _fields_ = [("num_views", C.c_int32), ("width", C.c_int32), ("height", C.c_int32),
                ("visible_capacity", C.c_int32),
                ("num_gaussians", C.c_int64), ("view_gauss_begin", C.POINTER(C.c_int64)),
                ("view_gauss_count", C.POINTER(C.c_int64)), ("cameras", C.c_void_p),
                ("key_capacity", C.c_int64), ("params", gs_params)]


class gs_gaussians(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacities", C.c_void_p), ("colors", C.c_void_p)]


class gs_image(C.Structure):
    _fields_ = [("rgb", C.c_void_p), ("depth", C.c_void_p), ("alpha", C.c_void_p), ("final_T", C.c_void_p),
                ("last_idx", C.c_void_p)]


class gs_image_grad(C.Structure):
    _fields_ = [("d_rgb", C.c_void_p), ("d_depth", C.c_void_p), ("d_alpha", C.c_void_p)]


class gs_grads(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacities", C.c_void_p), ("colors", C.c_void_p)]


class gs_ws_view(C.Structure):
    _fields_ = [("proj", C.c_void_p), ("tiles_touched", C.c_void_p), ("sorted_keys", C.c_void_p),
                ("sorted_vals", C.c_void_p), ("tile_ranges", C.c_void_p), ("grad2d", C.c_void_p),
                ("num_keys", C.c_void_p), ("num_pairs", C.c_int64), ("num_tiles", C.c_int64),
                ("sort_passes", C.c_int32), ("reserved", C.c_int32), ("pair_slot", C.c_void_p),
                ("visible_capacity", C.c_int64), ("claim_count", C.c_void_p), ("claim_list", C.c_void_p)]


class gs_stats(C.Structure):
    _fields_ = [("num_keys", C.c_int64), ("fwd_pairs", C.c_int64), ("bwd_pairs", C.c_int64),
                ("num_visible", C.c_int64)]


class gs_gaussian_arrays(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacities", C.c_void_p), ("colors", C.c_void_p)]


class gs_view_adam_state(C.Structure):
    _fields_ = [("cameras", C.c_void_p), ("expo", C.c_void_p), ("m", C.c_void_p), ("v", C.c_void_p),
                ("step", C.c_void_p)]


class gs_sim3(C.Structure):
    _fields_ = [("q", C.c_float * 4), ("t", C.c_float * 3), ("s", C.c_float)]


class gs_l1_target(C.Structure):
    _fields_ = [("rgb_t", C.c_void_p), ("depth_t", C.c_void_p), ("w_rgb", C.c_float), ("w_depth", C.c_float),
                ("d_rgb", C.c_void_p), ("d_depth", C.c_void_p), ("loss", C.c_void_p)]


class gs_pho_edge(C.Structure):
    _fields_ = [("src_image", C.c_int32), ("tgt_image", C.c_int32), ("src_corr", C.c_int32), ("tgt_corr", C.c_int32),
                ("weight", C.c_float), ("reserved", C.c_float * 3)]


class gs_pho_params(C.Structure):
    _fields_ = [("stride", C.c_int32), ("huber_delta", C.c_float), ("near_plane", C.c_float),
                ("reserved", C.c_int32)]


class gs_adam_state(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("opacities", C.c_void_p), ("colors", C.c_void_p),
                ("m", C.c_void_p), ("v", C.c_void_p), ("step", C.c_void_p)]


_P = C.c_void_p
_SIGS = {
    "gs_error_string": (C.c_char_p, [C.c_int]),
    "gs_version": (C.c_int, [C.POINTER(C.c_int)] * 3),
    "gs_default_params": (None, [C.POINTER(gs_params)]),
    "gs_workspace_size": (C.c_int, [C.POINTER(gs_problem), C.POINTER(C.c_size_t)]),
    "gs_workspace_init": (C.c_int, [C.POINTER(gs_problem), _P, _P]),
    "gs_workspace_view": (C.c_int, [C.POINTER(gs_problem), _P, C.POINTER(gs_ws_view)]),
    "gs_check_status": (C.c_int, [C.POINTER(gs_problem), _P, _P, C.POINTER(C.c_int64)]),
    "gs_read_stats": (C.c_int, [C.POINTER(gs_problem), _P, _P, C.POINTER(gs_stats)]),
    "gs_project": (C.c_int, [C.POINTER(gs_problem), C.POINTER(gs_gaussians), _P, _P]),
    "gs_bin_sort": (C.c_int, [C.POINTER(gs_problem), _P, _P]),
    "gs_render_fwd": (C.c_int, [C.POINTER(gs_problem), _P, C.POINTER(gs_image), _P]),
    "gs_render_fwd_l1": (C.c_int, [C.POINTER(gs_problem), _P, C.POINTER(gs_image), C.POINTER(gs_l1_target), _P]),
    "gs_render_bwd": (C.c_int, [C.POINTER(gs_problem), C.POINTER(gs_gaussians), _P, C.POINTER(gs_image),
                                C.POINTER(gs_image_grad), C.POINTER(gs_grads), _P]),
    "gs_render_bwd_composite": (C.c_int, [C.POINTER(gs_problem), _P, C.POINTER(gs_image), C.POINTER(gs_image_grad),
                                          _P]),
    "gs_project_bwd": (C.c_int, [C.POINTER(gs_problem), C.POINTER(gs_gaussians), _P, C.POINTER(gs_grads), _P]),
    "gs_pose_grad": (C.c_int, [C.POINTER(gs_problem), _P, _P, _P]),
    "gs_check_guards": (C.c_int, [C.POINTER(gs_problem), _P, _P, C.POINTER(C.c_int32)]),
    "gs_checked_build": (C.c_int32, []),
    "gs_loss_normal": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, _P, _P, _P, C.c_float, _P, _P, _P]),
    "gs_loss_l1": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, _P, _P, _P, _P, C.c_float, C.c_float, _P, _P, _P,
                             _P]),
    "gs_ssim_scratch_size": (C.c_size_t, [C.c_int32, C.c_int32, C.c_int32]),
    "gs_loss_l1_ssim": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, _P, _P, C.c_float, C.c_float, _P, _P, _P, _P]),
    "gs_loss_l1_ssim_noalloc": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, _P, _P, C.c_float, C.c_float, _P, _P,
                                          _P]),
    "gs_adam_step": (C.c_int, [C.c_int64, C.POINTER(gs_adam_state), C.POINTER(gs_grads),
                               C.POINTER(C.c_float), C.c_int32, _P]),
"gs_sim3_apply": (C.c_int, [C.c_int64, C.POINTER(gs_gaussians), C.POINTER(gs_sim3), C.POINTER(gs_gaussian_arrays),
                                _P]),
    "gs_voxset_bytes": (C.c_size_t, [C.c_int64]),
    "gs_voxset_clear": (C.c_int, [_P, C.c_int64, _P]),
    "gs_voxset_status": (C.c_int, [_P, _P, C.POINTER(C.c_int64), C.c_int64]),
    "gs_voxset_add_boxes": (C.c_int, [_P, C.c_int64, C.c_int64, _P, _P, C.c_float, C.c_float, _P]),
    "gs_voxset_add_rays": (C.c_int, [_P, C.c_int64, C.c_int32, C.c_int32, C.c_int32, _P, _P, C.c_int32, C.c_float,
                                     _P]),
    "gs_voxset_keep": (C.c_int, [C.c_int64, _P, _P, C.c_int64, _P, C.c_int64, C.c_float, _P, _P]),
    "gs_default_pho_params": (gs_pho_params, []),
    "gs_pho_scratch_size": (C.c_size_t, [C.c_int32]),
    "gs_pho_residual": (C.c_int, [C.c_int32, _P, C.c_int32, C.c_int32, C.c_int32, _P, _P, _P, C.c_int32, _P,
                                  C.POINTER(gs_pho_params), _P, _P, _P, _P, _P, C.c_size_t, _P]),
    "gs_adam_step_reg": (C.c_int, [C.c_int64, C.POINTER(gs_adam_state), C.POINTER(gs_grads), C.POINTER(C.c_float),
                                   C.c_float, C.c_int32, _P, _P]),
    "gs_refine_scratch_size": (C.c_size_t, [C.c_int32, C.c_int32, C.c_int32]),
    "gs_loss_refine": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, _P, _P, _P, _P, _P, C.c_float, C.c_float,
                                 C.c_float, _P, _P, _P, _P, _P, _P]),
    "gs_prune_scratch_size": (C.c_size_t, [C.c_int64]),
    "gs_prune": (C.c_int, [C.c_int64, C.POINTER(gs_gaussians), C.c_float, C.POINTER(gs_gaussian_arrays), _P, _P, _P]),
    "gs_view_adam_step": (C.c_int, [C.c_int32, C.POINTER(gs_view_adam_state), _P, _P, C.c_float, C.c_float, _P]),
    "gs_grads_zero": (C.c_int, [C.c_int64, C.POINTER(gs_grads), _P]),
    "gs_launch_count": (C.c_int64, []),
    "gs_debug_expf": (C.c_int, [_P, _P, _P, C.c_int64, _P]),
    "gs_debug_scan_scratch_size": (C.c_size_t, [C.c_int64]),
    "gs_debug_scan_timeout": (C.c_int, [_P, C.c_int64, C.c_int32, _P, C.POINTER(C.c_int64)]),
}

_lib = None


def variant() -> str:
    """'checked' when GS_LIBGS_VARIANT=checked selects the bounds-checked build, else 'release'."""
    return "checked" if os.environ.get("GS_LIBGS_VARIANT", "") == "checked" else "release"


def lib_path() -> str:
    name = "libgs_checked.so" if variant() == "checked" else "libgs.so"
    return os.path.join(_HERE, "_build", name)


def load(build_if_missing: bool = True):
    """Load libgs.so (building it first if it is absent and nvcc exists).  Raises on failure."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if build_if_missing:
        from . import build as _build
        try:
            path = _build.build(variant=variant())
        except Exception as e:  # noqa: BLE001
            if not os.path.exists(path):
                raise ImportError("libgs could not be built: %s" % e) from e
    if not os.path.exists(path):
        raise ImportError("libgs.so not found at %s (run __graft_entry__.build())" % path)
    L = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def error_string(code: int) -> str:
    try:
        return load(build_if_missing=False).gs_error_string(code).decode()
    except Exception:  # noqa: BLE001
        return "error %d" % code


def check(code: int, what: str):
    if code != GS_OK:
        raise GsError(code, what)


def header_symbols() -> list:
    """Names of the functions declared in include/gs.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", text)))
