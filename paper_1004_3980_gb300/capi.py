"""ctypes declarations of the C ABI in include/zoom.h (argument marshalling
only).  Importing this module loads libzoom.so and raises if it is missing:
there is no fallback implementation."""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libzoom.so")

ZOOM_OK = 0
STATUS_NAMES = {0: "ZOOM_OK", 1: "ZOOM_ERR_INVALID_ARG", 2: "ZOOM_ERR_OOM", 3: "ZOOM_ERR_CUDA",
                4: "ZOOM_ERR_TIMEOUT", 5: "ZOOM_ERR_UNSUPPORTED", 6: "ZOOM_ERR_STATE",
                7: "ZOOM_ERR_IO", 8: "ZOOM_ERR_DEVICE"}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


class Degradation(C.Structure):
    _fields_ = [("scale", C.c_int32), ("lr_patch", C.c_int32), ("blur_sigma", C.c_double),
                ("feature", C.c_int32)]


class LshParams(C.Structure):
    _fields_ = [("L", C.c_int32), ("k", C.c_int32), ("w", C.c_float),
                ("min_table_hits", C.c_int32), ("max_candidates", C.c_int32),
                ("proj_dist", C.c_int32), ("seed", C.c_uint64)]


class UpscaleParams(C.Structure):
    _fields_ = [("K", C.c_int32), ("reg_rel", C.c_float), ("bp_iters", C.c_int32),
                ("sigma_spatial", C.c_float), ("sigma_range", C.c_float), ("bp_radius", C.c_int32),
                ("precision", C.c_int32), ("rerank_mult", C.c_int32),
                ("fp64_cond_threshold", C.c_double), ("search", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("n_queries", C.c_int64), ("mean_bucket_sum", C.c_double),
                ("max_bucket_sum", C.c_int64), ("n_empty", C.c_int64),
                ("n_padded_queries", C.c_int64), ("n_fp64_solves", C.c_int64),
                ("n_exact_match", C.c_int64), ("n_filter_fallback", C.c_int64),
                ("ms_total", C.c_double), ("ms_stage", C.c_double * 8)]


_vp, _i32, _i64, _f = C.c_void_p, C.c_int32, C.c_int64, C.c_float
_P = C.POINTER

# name -> (restype, argtypes); the exported symbols of include/zoom.h
SIGNATURES = {
    "zoom_ctx_create": (C.c_int, [C.c_int, _P(Allocator), _P(_vp)]),
    "zoom_ctx_destroy": (None, [_vp]),
    "zoom_status_string": (C.c_char_p, [C.c_int]),
    "zoom_last_error": (C.c_char_p, []),
    "zoom_build_dictionary": (C.c_int, [_vp, _P(_vp), _P(_i32), _P(_i32), _i32, _P(Degradation),
                                        _i64, _P(_i32), C.c_uint64, _vp, _P(_vp)]),
    "zoom_lsh_draws": (C.c_int, [_P(LshParams), _i32, _vp, _vp]),
    "zoom_sample_positions": (C.c_int, [C.c_uint64, _i32, _P(_i32), _P(_i32), _i32, _i64, _vp]),
    "zoom_dict_destroy": (None, [_vp]),
    "zoom_dict_export": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "zoom_dict_info": (C.c_int, [_vp, _P(_i64), _P(_i32), _P(_i32), _P(C.c_double), _P(_i32), _P(_i32)]),
    "zoom_dict_save": (C.c_int, [_vp, C.c_char_p, _vp]),
    "zoom_sample_crops": (C.c_int, [_vp, _P(_vp), _P(_i32), _P(_i32), _i32, _vp, _i32, _i32, _i32, _vp, _vp,
                                    _vp]),
    "zoom_dict_load": (C.c_int, [_vp, C.c_char_p, _vp, _P(_vp)]),
    "zoom_index_save": (C.c_int, [_vp, C.c_char_p, _vp]),
    "zoom_index_load": (C.c_int, [_vp, C.c_char_p, _vp, _P(_vp)]),
    "zoom_index_info": (C.c_int, [_vp, _P(LshParams)]),
    "zoom_export_params": (C.c_int, [_vp, _vp, _vp, _vp]),
    "zoom_build_index": (C.c_int, [_vp, _P(LshParams), _vp, _vp, _vp, _P(_vp)]),
    "zoom_index_destroy": (None, [_vp]),
    "zoom_index_export": (C.c_int, [_vp, _vp, _vp, _vp]),
    "zoom_upscale": (C.c_int, [_vp, _vp, _i32, _i32, _i32, _P(UpscaleParams), _vp, _vp]),
    "zoom_query": (C.c_int, [_vp, _vp, _i32, _i32, _P(UpscaleParams), _vp, _vp, _vp, _vp, _vp,
                             _vp, _vp]),
    "zoom_reconstruct": (C.c_int, [_vp, _vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp]),
    "zoom_backproject": (C.c_int, [_vp, _P(Degradation), _vp, _i32, _i32, _P(UpscaleParams), _vp,
                                   _vp]),
    "zoom_get_stats": (C.c_int, [_vp, _vp, _P(Stats)]),
    "zoom_sync_status": (C.c_int, [_vp, _vp]),
    "zoom_set_fault_injection": (C.c_int, [_vp, C.c_int32, C.c_uint64]),
    "zoom_set_stage_timing": (C.c_int, [_vp, C.c_int32]),
    "zoom_backproject_noalloc": (C.c_int, [C.c_int, _P(Degradation), _vp, _i32, _i32,
                                           _P(UpscaleParams), _vp, _vp]),
    "zoom_upscale_batch": (C.c_int, [_P(_vp), _i32, _i32, _P(_vp), _P(_i32), _P(_i32), _P(_i32),
                                     _P(UpscaleParams), _P(_vp), _vp, _P(_f)]),
    "zoom_batch_release": (C.c_int, [_vp]),
    "zoom_degrade": (C.c_int, [_vp, _P(Degradation), _vp, _i32, _i32, _vp, _vp]),
    "zoom_degrade_adjoint": (C.c_int, [_vp, _P(Degradation), _vp, _i32, _i32, _vp, _vp]),
    "zoom_reconstruct_with": (C.c_int, [_vp, _vp, _i32, _vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp]),
    "zoom_reconstruct_adjoint": (C.c_int, [_vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp, _i32, _vp, _vp]),
    "zoom_backward": (C.c_int, [_vp, _vp, _i32, _i32, _vp, _vp, _i32, _f, _f, _vp, _vp, _i32, _vp,
                                _P(C.c_double), _vp]),
}


class ZoomError(RuntimeError):
    def __init__(self, fn: str, status: int, detail: str):
        self.status = status
        super().__init__(f"{fn} -> {STATUS_NAMES.get(status, status)}: {detail}")


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_1004_3980_gb300.build` "
                          "(there is no fallback implementation)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_LIB = None


def lib() -> C.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = load()
    return _LIB


def check(name: str, status: int) -> None:
    if status != ZOOM_OK:
        raise ZoomError(name, status, lib().zoom_last_error().decode())


def call(name: str, *args) -> None:
    check(name, getattr(lib(), name)(*args))
