"""ctypes binding of ``libelas_gb300.so`` (the C-ABI in include/elas_gb300.h).

Argument marshalling only: tensors are checked for device, dtype, shape and
contiguity, their data pointers and the current CUDA stream are passed to the
C entry point of the same name, and a non-OK status raises ``ElasError``.
Every step of the path runs in the library's CUDA kernels (the triangulation
in its host code); nothing here computes any part of the method, and there is
no fallback: if the library is missing, loading fails loudly.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libelas_gb300.so")

STATUS = {0: "ELAS_OK", 1: "ELAS_ERR_INVALID_ARG", 2: "ELAS_ERR_CUDA", 3: "ELAS_ERR_CAPACITY",
          4: "ELAS_ERR_TIMEOUT", 5: "ELAS_ERR_NO_MEMORY", 6: "ELAS_ERR_INTERNAL"}

FLAG_PRIOR_OFF = 1
FLAG_FULL_RANGE = 2
FLAG_REDUNDANCY_OFF = 4


class ElasError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class Params(C.Structure):
    """Mirror of ``elas_params`` (field order and types must match)."""
    _fields_ = [
        ("disp_min", C.c_int32), ("disp_max", C.c_int32),
        ("support_threshold", C.c_float), ("support_texture", C.c_int32),
        ("candidate_stepsize", C.c_int32),
        ("incon_window_size", C.c_int32), ("incon_threshold", C.c_int32),
        ("incon_min_support", C.c_int32), ("redun_max_dist", C.c_int32),
        ("grid_size", C.c_int32),
        ("beta", C.c_float), ("gamma", C.c_float), ("sigma", C.c_float),
        ("sradius", C.c_int32), ("match_texture", C.c_int32), ("lr_threshold", C.c_int32),
        ("ipol_gap_width", C.c_int32), ("filter_adaptive_mean", C.c_int32),
        ("test_flags", C.c_uint32),
        ("census_support_w", C.c_int32), ("census_dense_w", C.c_int32),
        ("support_downsample", C.c_int32),
    ]


class PipelineStats(C.Structure):
    _fields_ = [("n_support", C.c_int32), ("n_tri_left", C.c_int32),
                ("n_tri_right", C.c_int32), ("triangulate_ms", C.c_double), ("stage_ms", C.c_float * 6)]


class BatchConfig(C.Structure):
    _fields_ = [("desc_tile_rows", C.c_int32), ("support_warps", C.c_int32),
                ("dense_threads_per_pixel", C.c_int32), ("use_graph", C.c_int32),
                ("dense_pixels_per_thread", C.c_int32), ("dense_fused", C.c_int32)]


class ServerConfig(C.Structure):
    _fields_ = [("lanes", C.c_int32), ("max_wave", C.c_int32), ("max_slots", C.c_int32), ("plain", C.c_int32),
                ("hbm_budget_bytes", C.c_uint64), ("hbm_reserve_bytes", C.c_uint64)]


class ServerResult(C.Structure):
    _fields_ = [("id", C.c_uint64), ("status", C.c_int32), ("n_support", C.c_int32), ("wave_size", C.c_int32),
                ("pad", C.c_int32), ("t_submit_ms", C.c_double), ("t_start_ms", C.c_double),
                ("t_done_ms", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("waves", C.c_int64),
                ("slots_created", C.c_int64), ("slots_released", C.c_int64), ("slots_in_use", C.c_int32),
                ("max_wave_seen", C.c_int32), ("slot_bytes", C.c_uint64), ("hbm_budget_bytes", C.c_uint64)]


_P, _I, _Z = C.c_void_p, C.c_int32, C.c_size_t

# name -> (restype, argtypes), exactly the declarations of include/*.h
SIGNATURES = {
    "elas_params_default": (C.c_int, [_P]),
    "elas_last_error": (C.c_char_p, []),
    "elas_version": (C.c_char_p, []),
    "elas_descriptors": (C.c_int, [_P, _P, _I, _I, _I, _P, _P, _P]),
    "elas_census": (C.c_int, [_P, _P, _I, _I, _I, _I, _I, _P, _P, _P]),
    "elas_support_workspace_bytes": (_Z, [_I, _I, _P]),
    "elas_support_points": (C.c_int, [_P, _P, _I, _I, _P, _P, _P, _I, _P, _P, _P, _P, _Z, _P]),
    "elas_support_points_static": (C.c_int, [_P, _P, _I, _I, _P, _P, _P, _I, _P, _P, _P, _P]),
    "elas_triangulate": (C.c_int, [_P, _I, _I, _P, _I, _P]),
    "elas_triangulate_device_workspace_bytes": (_Z, [_I, _I, _I]),
    "elas_triangulate_device": (C.c_int, [_P, _P, _I, _I, _I, _I, _P, _I, _P, _P, _Z, _P]),
    "elas_plane_prior_workspace_bytes": (_Z, [_I]),
    "elas_plane_prior": (C.c_int, [_P, _I, _P, _I, _I, _I, _I, _P, _P, _P, _Z, _P]),
    "elas_dense_argmin": (C.c_int, [_P, _P, _I, _I, _P, _P, _P, _I, _P, _P]),
    "elas_dense_workspace_bytes": (_Z, [_I, _I, _P]),
    "elas_dense_match": (C.c_int, [_P, _P, _I, _I, _P, _P, _I, _P, _I, _P, _I, _P, _P, _P, _P,
                                   _P, _Z, _P]),
    "elas_lr_check": (C.c_int, [_P, _P, _I, _I, _I, _P, _P, _P]),
    "elas_postprocess_workspace_bytes": (_Z, [_I, _I]),
    "elas_postprocess": (C.c_int, [_P, _I, _I, _P, _P, _P, _Z, _P]),
    "elas_median": (C.c_int, [_P, _I, _I, _I, _P, _P]),
    "elas_speckle_workspace_bytes": (C.c_size_t, [_I, _I]),
    "elas_workspace_bytes": (C.c_size_t, [_I, _I, _P]),
    "elas_speckle": (C.c_int, [_P, _I, _I, _I, _I, _P, _P, C.c_size_t, _P]),
    "elas_pipeline_create": (C.c_int, [_I, _I, _P, _P]),
    "elas_pipeline_run": (C.c_int, [_P, _P, _P, _I, _P, _P, _P, _P]),
    "elas_pipeline_run_host": (C.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "elas_pipeline_set_triangulation": (C.c_int, [_P, _I]),
    "elas_pipeline_set_profiling": (C.c_int, [_P, _I]),
    "elas_pipeline_set_graph": (C.c_int, [_P, _I]),
    "elas_pipeline_stats_get": (C.c_int, [_P, _P]),
    "elas_pipeline_destroy": (None, [_P]),
    "elas_batch_create": (C.c_int, [_I, _P, _P, _P, _P]),
    "elas_batch_get_config": (C.c_int, [_P, _P]),
    "elas_batch_set_config": (C.c_int, [_P, _P]),
    "elas_batch_run": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "elas_batch_run_host": (C.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "elas_batch_stats": (C.c_int, [_P, _P, _P, _P]),
    "elas_batch_tune": (C.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "elas_batch_profile": (C.c_int, [_P, _P, _P]),
    "elas_batch_device_bytes": (_Z, [_P]),
    "elas_batch_destroy": (None, [_P]),
    "elas_server_config_default": (C.c_int, [_P]),
    "elas_slot_device_bytes": (_Z, [_I, _I, _P]),
    "elas_server_create": (C.c_int, [_P, _P]),
    "elas_server_submit": (C.c_int, [_P, C.c_uint64, _I, _I, _P, _P, _P, _P, _P]),
    "elas_server_poll": (C.c_int32, [_P, _P, _I, _I]),
    "elas_server_now_ms": (C.c_double, [_P]),
    "elas_server_stats_get": (C.c_int, [_P, _P]),
    "elas_server_drain": (C.c_int, [_P, _I]),
    "elas_server_inject_alloc_failures": (C.c_int, [_P, _I]),
    "elas_server_destroy": (None, [_P]),
    "elas_probe_sad16": (C.c_int, [_I, _I, _I, _I, _P, _P]),
}

_lib = None


def lib():
    """Loads the library (building it first only if it is absent and nvcc is
    available); raises if it cannot be loaded."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            from . import build as _build
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libelas_gb300.so is missing: run paper_1802_07210_gb300/build.py")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status):
    if status != 0:
        raise ElasError(status, lib().elas_last_error().decode())


def params(**kw) -> Params:
    p = Params()
    check(lib().elas_params_default(C.byref(p)))
    for k, v in kw.items():
        if k == "flags":
            k = "test_flags"
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def as_params(prm) -> Params:
    if prm is None:
        return params()
    if isinstance(prm, dict):
        return params(**prm)
    return prm


def np_ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)
