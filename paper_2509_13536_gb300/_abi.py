"""ctypes declarations of include/memgs.h (argument marshalling only).

The names mirror the C ABI one to one.  Loading fails loudly when libmemgs.so has not
been built: there is no fallback implementation of any entry point.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

MGS_MAX_VIEWS = 32
MGS_SORT_NOALLOC_MAX = 1 << 20
MGS_OK, MGS_ERR_INVALID, MGS_ERR_WORKSPACE, MGS_ERR_CUDA, MGS_ERR_TIMEOUT, MGS_ERR_UNSUPPORTED = range(6)
MGS_F32, MGS_F16, MGS_BF16 = 0, 1, 2
STATUS_NAMES = {0: "MGS_OK", 1: "MGS_ERR_INVALID", 2: "MGS_ERR_WORKSPACE", 3: "MGS_ERR_CUDA",
                4: "MGS_ERR_TIMEOUT", 5: "MGS_ERR_UNSUPPORTED"}

EXPORTS = ["mgs_render_workspace_size", "mgs_render", "mgs_render_backward", "mgs_project",
           "mgs_voxel_merge_workspace_size", "mgs_voxel_merge", "mgs_adam_step", "mgs_l1_loss_grad",
           "mgs_sort_workspace_size", "mgs_sort_pairs", "mgs_last_error", "mgs_version",
           "mgs_launch_count", "mgs_profile_enable", "mgs_profile_read", "mgs_render_stats",
           "mgs_sort_pairs_noalloc", "mgs_server_create", "mgs_server_add_scene", "mgs_server_submit",
           "mgs_server_poll", "mgs_server_clock", "mgs_server_destroy", "mgs_mapping_loss_workspace_size",
           "mgs_mapping_loss", "mgs_iso_loss_workspace_size", "mgs_iso_loss", "mgs_merge_stats",
           "mgs_patch_grid_workspace_size", "mgs_patch_grid_capacity", "mgs_patch_grid_sample",
           "mgs_render_multi_workspace_size", "mgs_render_multi", "mgs_server_stats", "mgs_render_async",
           "mgs_voxel_merge_async"]


class mgs_gaussians(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32), ("attr_dtype", C.c_int32),
                ("geom_dtype", C.c_int32), ("quat_dtype", C.c_int32), ("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("sh", C.c_void_p), ("birth", C.c_void_p)]


mgs_gaussians_mut = mgs_gaussians  # same layout, non-const pointers


class mgs_camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("near_z", C.c_float), ("reserved", C.c_int32)]


class mgs_image(C.Structure):
    _fields_ = [("rgb", C.c_void_p), ("depth", C.c_void_p), ("alpha", C.c_void_p)]


class mgs_grads(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("means", "log_scales", "quats", "opacity_logit", "sh",
                                          "grad_stat", "vis_count")] + \
               [("overwrite", C.c_int32), ("reserved", C.c_int32)]


class mgs_server_config(C.Structure):
    _fields_ = [("n_slots", C.c_int32), ("max_batch_views", C.c_int32), ("device", C.c_int32),
                ("reserved", C.c_int32), ("arena", C.c_void_p), ("arena_bytes", C.c_size_t)]


class mgs_merge_params(C.Structure):
    _fields_ = [("chi2", C.c_float), ("grad_tau", C.c_float), ("kf_min", C.c_int32),
                ("kf_max", C.c_int32), ("grad_stat", C.c_void_p), ("kf_id", C.c_void_p),
                ("vis_count", C.c_void_p), ("greedy", C.c_int32), ("solver", C.c_int32)]


class mgs_pg_params(C.Structure):
    _fields_ = [("patch", C.c_int32), ("min_keypoints", C.c_int32), ("grid", C.c_int32),
                ("reserved", C.c_int32)]


_lock = threading.Lock()
_lib = None


class MemgsError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def lib_path() -> str:
    """The in-tree build, or the library named by MEMGS_LIB (a deployment override)."""
    return os.environ.get("MEMGS_LIB") or _build.LIB


def load():
    """Load libmemgs.so (built in-tree by ``build.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            raise ImportError(f"libmemgs.so is not built ({path}); run paper_2509_13536_gb300.build.build()")
        L = C.CDLL(path)
        P, I64, I32, F, SZ = C.c_void_p, C.c_int64, C.c_int32, C.c_float, C.c_size_t
        sig = {
            "mgs_render_workspace_size": (SZ, [I64, P, I32, I64]),
            "mgs_render": (C.c_int, [P, P, I32, P, P, SZ, P, P]),
            "mgs_render_multi_workspace_size": (SZ, [P, I32, P, P, I32, I64]),
            "mgs_render_multi": (C.c_int, [P, I32, P, P, I32, P, P, SZ, P, P]),
            "mgs_render_async": (C.c_int, [P, P, I32, P, P, SZ, P, P]),
            "mgs_voxel_merge_async": (C.c_int, [P, F, P, P, P, P, P, P, SZ, P]),
            "mgs_render_backward": (C.c_int, [P, P, I32, P, P, SZ, P, P]),
            "mgs_project": (C.c_int, [P, P, P, P, P, P, P, P, P]),
            "mgs_voxel_merge_workspace_size": (SZ, [I64]),
            "mgs_voxel_merge": (C.c_int, [P, F, P, P, P, P, P, P, SZ, P]),
            "mgs_adam_step": (C.c_int, [P, P, P, P, F, F, F, F, I32, I32, P]),
            "mgs_l1_loss_grad": (C.c_int, [P, P, I64, F, P, P, P]),
            "mgs_sort_workspace_size": (SZ, [I64]),
            "mgs_mapping_loss_workspace_size": (SZ, [I32, I32, I32]),
            "mgs_mapping_loss": (C.c_int, [I32, I32, I32, P, P, P, F, F, P, P, SZ, P]),
            "mgs_iso_loss_workspace_size": (SZ, [I64]),
            "mgs_iso_loss": (C.c_int, [P, F, P, P, P, SZ, P]),
            "mgs_merge_stats": (None, [P]),
            "mgs_patch_grid_workspace_size": (SZ, [I32, I32, P]),
            "mgs_patch_grid_capacity": (I64, [I32, I32, P]),
            "mgs_patch_grid_sample": (C.c_int, [P, I32, P, P, P, P, P, P, I64, P, P, SZ, P]),
            "mgs_sort_pairs": (C.c_int, [P, P, P, I64, I32, I32, P, SZ, P]),
            "mgs_sort_pairs_noalloc": (C.c_int, [P, P, P, I64, I32, I32, P]),
            "mgs_server_create": (C.c_int, [P, P]),
            "mgs_server_add_scene": (C.c_int, [P, P, P]),
            "mgs_server_submit": (C.c_int, [P, I32, P, P, I64, C.c_double]),
            "mgs_server_poll": (I32, [P, I32, P, P, P, P, P, C.c_double]),
            "mgs_server_clock": (C.c_double, []),
            "mgs_server_stats": (C.c_int, [P, P]),
            "mgs_server_destroy": (C.c_int, [P]),
            "mgs_launch_count": (C.c_uint64, []),
            "mgs_profile_enable": (None, [I32]),
            "mgs_profile_read": (I32, [I32, P, P, P]),
            "mgs_render_stats": (C.c_int, [P, P, I32, P, SZ, P, P]),
            "mgs_last_error": (C.c_char_p, []),
            "mgs_version": (C.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def check(status: int, where: str):
    if status != MGS_OK:
        msg = load().mgs_last_error().decode(errors="replace")
        raise MemgsError(status, where, msg)
