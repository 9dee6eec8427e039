"""ctypes declarations of the C ABI in include/gs.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os
import threading

_lock = threading.Lock()
_lib = None

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libgs.so")


class gs_camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("near_z", C.c_float)]


class gs_gaussians(C.Structure):
    _fields_ = [("means", C.c_void_p), ("scales", C.c_void_p), ("quats", C.c_void_p), ("opacity", C.c_void_p),
                ("sh", C.c_void_p), ("P", C.c_int64), ("sh_degree", C.c_int32), ("activated", C.c_int32),
                ("sh_half", C.c_int32), ("reserved", C.c_int32)]


class gs_render_opts(C.Structure):
    _fields_ = [("bg", C.c_float * 3), ("tau", C.c_float), ("alpha_max", C.c_float), ("T_min", C.c_float),
                ("dilation", C.c_float), ("cap_3sigma", C.c_int32), ("clamp_fov", C.c_int32),
                ("intersect", C.c_int32)]


class gs_frame_stats(C.Structure):
    _fields_ = [("pairs", C.c_int64), ("visible", C.c_int64), ("pair_capacity", C.c_int64), ("status", C.c_int32),
                ("width", C.c_int32), ("height", C.c_int32), ("tiles_x", C.c_int32), ("tiles_y", C.c_int32),
                ("sort_passes", C.c_int32), ("culled_in", C.c_int64), ("evaluations", C.c_int64),
                ("contributions", C.c_int64), ("kernels", C.c_int32), ("pad", C.c_int32)]


class gs_gaussian_grads(C.Structure):
    _fields_ = [("means", C.c_void_p), ("scales", C.c_void_p), ("quats", C.c_void_p), ("opacity", C.c_void_p),
                ("sh", C.c_void_p)]


class gs_server_cfg(C.Structure):
    _fields_ = [("slots", C.c_int32), ("max_batch", C.c_int32), ("pair_capacity", C.c_int64),
                ("max_gaussians", C.c_int64), ("max_width", C.c_int32), ("max_height", C.c_int32),
                ("sort_mode", C.c_int32), ("blend_variant", C.c_int32), ("plain", C.c_int32), ("batch_pixels", C.c_int32),
                ("overlap_pending", C.c_int32), ("fifo_load_pct", C.c_int32)]


class gs_request_stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("batch_size", C.c_int32), ("arrival_s", C.c_double),
                ("admit_s", C.c_double), ("done_s", C.c_double), ("pairs", C.c_int64)]


class gs_server_stats(C.Structure):
    _fields_ = [("completed", C.c_int64), ("batches", C.c_int64), ("batched_requests", C.c_int64),
                ("pending", C.c_int64)]


class gs_tuning(C.Structure):
    _fields_ = [("blend_variant", C.c_int32), ("sort_mode", C.c_int32), ("sort_algo", C.c_int32),
                ("reserved", C.c_int32 * 5)]


class gs_alu_peaks(C.Structure):
    _fields_ = [("fma_tops", C.c_double), ("ex2_tops", C.c_double), ("fma_ms", C.c_double), ("ex2_ms", C.c_double),
                ("sm_count", C.c_int32), ("pad", C.c_int32)]


_vp = C.c_void_p
ROUTER_SUBMIT = C.CFUNCTYPE(C.c_int32, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                            C.c_double, C.POINTER(C.c_uint64))
ROUTER_WAIT = C.CFUNCTYPE(C.c_int32, C.c_void_p, C.c_int32, C.c_uint64, C.c_int32, C.c_void_p)


class gs_router_backend(C.Structure):
    _fields_ = [("submit", ROUTER_SUBMIT), ("wait", ROUTER_WAIT), ("user", C.c_void_p)]

_pp = C.POINTER(C.c_void_p)
_st = C.c_int32

# name -> (restype, argtypes); every symbol declared in include/gs.h
PROTOTYPES = {
    "gs_last_error": (C.c_char_p, []),
    "gs_version": (C.c_int32, []),
    "gs_default_opts": (_st, [C.POINTER(gs_render_opts)]),
    "gs_context_create": (_st, [C.c_int32, _pp]),
    "gs_context_destroy": (_st, [_vp]),
    "gs_scene_create": (_st, [_vp, C.POINTER(gs_gaussians), _vp, _pp]),
    "gs_scene_update": (_st, [_vp, C.POINTER(gs_gaussians), _vp]),
    "gs_scene_destroy": (_st, [_vp]),
    "gs_scene_size": (C.c_int64, [_vp]),
    "gs_frame_create": (_st, [_vp, C.c_int64, C.c_int64, C.c_int32, C.c_int32, _pp]),
    "gs_frame_destroy": (_st, [_vp]),
    "gs_frame_bytes": (C.c_int64, [_vp]),
    "gs_preprocess": (_st, [_vp, _vp, C.POINTER(gs_camera), C.POINTER(gs_render_opts), _vp]),
    "gs_sort": (_st, [_vp, _vp]),
    "gs_ranges": (_st, [_vp, _vp]),
    "gs_blend": (_st, [_vp, C.POINTER(gs_render_opts), _vp, _vp, _vp, _vp]),
    "gs_render": (_st, [_vp, _vp, C.POINTER(gs_camera), C.POINTER(gs_render_opts), _vp, _vp, _vp, _vp]),
    "gs_frame_use_graph": (_st, [_vp, C.c_int32]),
    "gs_render_batch": (_st, [_vp, C.c_int32, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "gs_render_backward": (_st, [_vp, _vp, _vp, _vp, _vp, C.POINTER(gs_gaussian_grads), C.c_int32, _vp]),
    "gs_frame_enable_timing": (_st, [_vp, C.c_int32]),
    "gs_frame_set_tuning": (_st, [_vp, C.POINTER(gs_tuning)]),
    "gs_frame_get_tuning": (_st, [_vp, C.POINTER(gs_tuning)]),
    "gs_frame_set_counting": (_st, [_vp, C.c_int32]),
    "gs_autotune": (_st, [_vp, _vp, _vp, C.c_int32, C.POINTER(gs_render_opts), C.c_char_p, C.POINTER(gs_tuning),
                          _vp]),
    "gs_frame_stage_ms": (_st, [_vp, C.POINTER(C.c_float)]),
    "gs_measure_alu_peaks": (_st, [C.c_int32, C.c_double, C.POINTER(gs_alu_peaks)]),
    "gs_render_host": (_st, [_vp, _vp, C.POINTER(gs_camera), C.POINTER(gs_render_opts), _vp, _vp, _vp, _vp]),
    "gs_frame_get_stats": (_st, [_vp, C.POINTER(gs_frame_stats), _vp]),
    "gs_frame_pairs": (_st, [_vp, C.c_int32, _vp, _vp, C.c_int64, C.POINTER(C.c_int64), _vp]),
    "gs_frame_ranges": (_st, [_vp, _vp, C.c_int64, _vp]),
    "gs_sort_pairs": (_st, [_vp, _vp, _vp, _vp, _vp, C.c_int64, C.c_int32, C.POINTER(C.c_int32), _vp]),
    "gs_clock_s": (C.c_double, []),
    "gs_server_hold": (_st, [_vp, C.c_int32]),
    "gs_router_create": (_st, [C.c_int32, C.POINTER(gs_router_backend), _pp]),
    "gs_router_create_on_servers": (_st, [C.c_int32, C.POINTER(C.c_void_p), _pp]),
    "gs_router_destroy": (_st, [_vp]),
    "gs_router_place_scene": (_st, [_vp, C.c_int32, C.c_int32, _vp]),
    "gs_router_submit": (_st, [_vp, C.c_int32, C.POINTER(gs_camera), C.POINTER(gs_render_opts), _vp, C.c_double,
                               C.POINTER(C.c_uint64)]),
    "gs_router_wait": (_st, [_vp, C.c_uint64, C.c_int32, C.POINTER(gs_request_stats), C.POINTER(C.c_int32)]),
    "gs_router_outstanding": (_st, [_vp, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "gs_default_server_cfg": (_st, [C.POINTER(gs_server_cfg)]),
    "gs_server_create": (_st, [_vp, C.POINTER(gs_server_cfg), _pp]),
    "gs_server_destroy": (_st, [_vp]),
    "gs_server_submit": (_st, [_vp, _vp, C.POINTER(gs_camera), C.POINTER(gs_render_opts), _vp, C.c_double,
                               C.POINTER(C.c_uint64)]),
    "gs_server_wait": (_st, [_vp, C.c_uint64, C.c_int32, C.POINTER(gs_request_stats)]),
    "gs_server_get_stats": (_st, [_vp, C.POINTER(gs_server_stats)]),
    "gs_sort_pairs_noalloc": (_st, [_vp, _vp, _vp, _vp, C.c_int64, C.c_int32, C.POINTER(C.c_int32), _vp]),
    "gs_eval_decision_math": (_st, [C.c_int32, _vp, _vp, C.c_int64, C.c_float, _vp]),
    "gs_sort_pairs_status": (_st, [_vp, _vp]),
    "gs_set_wait_limit": (_st, [C.c_uint32]),
    "gs_get_wait_limit": (C.c_uint32, []),
    "gs_sort_pairs_noalloc_status": (_st, [_vp]),
    "gs_frame_backward_ms": (_st, [_vp, C.POINTER(C.c_float)]),
}


def load(path: str | None = None):
    """Load libgs.so and attach the prototypes.  Raises if the library is missing: there is no
    fallback implementation."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"libgs.so not built ({p}); run paper_2408_07967_gb300.build.build()")
            L = C.CDLL(p)
            for name, (res, args) in PROTOTYPES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib
