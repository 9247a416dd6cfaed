"""ctypes declarations of include/occ.h and the loader of liboccreuse.so.

The library must exist (``build()`` makes it); there is no fallback of any kind.
OCC_LIB_VARIANT=counters (environment) loads the instrumented build instead (see
build.VARIANTS), which only measurement runs use.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from .build import build as _do_build, lib_path as _lib_path, up_to_date as _up_to_date

c_int32, c_int64, c_uint32, c_uint64 = C.c_int32, C.c_int64, C.c_uint32, C.c_uint64
c_float, c_double, c_void_p, c_char_p = C.c_float, C.c_double, C.c_void_p, C.c_char_p

OCC_OK = 0
STATUS_NAMES = {0: "OCC_OK", 1: "OCC_ERR_INVALID_ARG", 2: "OCC_ERR_CUDA", 3: "OCC_ERR_OOM",
                4: "OCC_ERR_TIMEOUT", 5: "OCC_ERR_UNSUPPORTED", 6: "OCC_ERR_DEVICE_CHECK",
                7: "OCC_ERR_BUSY", 8: "OCC_ERR_CANCELLED"}

OCC_EFFECT_AO, OCC_EFFECT_SHADOW = 0, 1
OCC_EST_NOREUSE, OCC_EST_BIASED, OCC_EST_UNBIASED, OCC_EST_BOXMEAN = 0, 1, 2, 3
OCC_EST_LIGHT_UNBIASED = 4
OCC_PAT_GROUP, OCC_PAT_BOX, OCC_PAT_OFFSETS, OCC_PAT_RANDOM = 0, 1, 2, 3
OCC_REC_FP32, OCC_REC_PACKED = 0, 1
OCC_GB_FP32, OCC_GB_PACKED = 0, 1
OCC_LAYOUT_LINEAR, OCC_LAYOUT_TILED = 0, 1
MAX_MEMBERS = 64


class occ_gbuffer(C.Structure):
    _fields_ = [("W", c_int32), ("H", c_int32), ("pos4", c_void_p), ("nrm4", c_void_p),
                ("format", c_int32), ("layout", c_int32), ("pitch_px", c_int64)]


class occ_rect_light(C.Structure):
    _fields_ = [("c", c_float * 3), ("eu", c_float * 3), ("ev", c_float * 3)]


class occ_occluders(C.Structure):
    _fields_ = [("W", c_int32), ("H", c_int32), ("format", c_int32), ("data", c_void_p),
                ("effect", c_int32), ("radius", c_float), ("light", occ_rect_light),
                ("seed", c_uint64), ("sample", c_uint32)]


class occ_pattern(C.Structure):
    _fields_ = [("kind", c_int32), ("gw", c_int32), ("gh", c_int32), ("n_offsets", c_int32),
                ("offsets_host", C.POINTER(c_int32)), ("radius_px", c_int32), ("seed", c_uint64)]


class occ_view(C.Structure):
    _fields_ = [("gb", occ_gbuffer), ("rec", occ_occluders), ("effect", c_int32),
                ("radius", c_float), ("light", occ_rect_light), ("seed", c_uint64),
                ("sample", c_uint32), ("pattern", occ_pattern), ("K", c_int32),
                ("estimator", c_int32), ("out", c_void_p)]


class occ_tuning(C.Structure):
    _fields_ = [("reuse_tile_rows", c_int32), ("reuse_window_path", c_int32),
                ("batch_ctas_per_sm", c_int32), ("fused_ao_path", c_int32),
                ("group_prefetch", c_int32), ("trace_path", c_int32),
                ("trace_ctas_per_sm", c_int32), ("trace_refill", c_int32),
                ("trace_order", c_int32)]


class occ_bvh_stats(C.Structure):
    _fields_ = [("num_tris", c_int64), ("num_nodes", c_int64), ("num_leaves", c_int64),
                ("depth", c_int32), ("max_leaf_tris", c_int32), ("bytes", c_int64),
                ("build_seconds", c_double)]


# include/occ_serve.h
class occ_sched_config(C.Structure):
    _fields_ = [("budget_bytes", c_int64), ("max_views_per_batch", c_int32),
                ("max_inflight", c_int32), ("max_queued", c_int32)]


class occ_sched_stats(C.Structure):
    _fields_ = [(f, c_int64) for f in ("queued", "inflight_batches", "reserved_bytes",
                                       "peak_reserved_bytes", "submitted", "admitted",
                                       "completed_batches", "expired", "refused")]


class occ_server_config(C.Structure):
    _fields_ = [("budget_bytes", c_int64), ("max_views_per_batch", c_int32),
                ("max_inflight", c_int32), ("max_queued", c_int32), ("poll_us", c_int32),
                ("batch_max_px", c_int64), ("batch_window_us", c_int64),
                ("inject_alloc_failures", c_int32), ("reserved", c_int32)]


class occ_request(C.Structure):
    _fields_ = [("W", c_int32), ("H", c_int32), ("effect", c_int32), ("radius", c_float),
                ("light", occ_rect_light), ("seed", c_uint64), ("sample", c_uint32),
                ("pattern", occ_pattern), ("K", c_int32), ("estimator", c_int32),
                ("packed", c_int32), ("camera", c_float * 10), ("eps", c_float),
                ("pos4_host", c_void_p), ("nrm4_host", c_void_p), ("out_host", c_void_p),
                ("out_device", c_void_p), ("deadline_ns", c_int64)]


class occ_result(C.Structure):
    _fields_ = [("id", c_uint64), ("status", c_int32), ("batch_views", c_int32),
                ("t_submit_ns", c_int64), ("t_admit_ns", c_int64), ("t_done_ns", c_int64)]


class occ_server_stats(C.Structure):
    _fields_ = [("sched", occ_sched_stats), ("budget_bytes", c_int64), ("batches", c_int64),
                ("views_batched", c_int64), ("views_single", c_int64),
                ("pool_reserved_bytes", c_int64)]


# name -> (restype, argtypes); every symbol declared in include/*.h
SIGNATURES = {
    "occ_create": (c_int32, [C.c_int, C.POINTER(c_void_p)]),
    "occ_destroy": (c_int32, [c_void_p]),
    "occ_last_error": (c_char_p, [c_void_p]),
    "occ_sync": (c_int32, [c_void_p, c_void_p]),
    "occ_version": (c_char_p, []),
    "occ_bvh_build": (c_int32, [c_void_p, c_void_p, c_int64, C.POINTER(c_void_p)]),
    "occ_bvh_free": (c_int32, [c_void_p, c_void_p]),
    "occ_bvh_info": (c_int32, [c_void_p, C.POINTER(occ_bvh_stats)]),
    "occ_gbuffer_pinhole": (c_int32, [c_void_p, c_void_p, c_void_p, c_float, c_int32, c_int32,
                                      c_void_p, c_void_p, c_void_p]),
    "occ_pack_gbuffer": (c_int32, [c_void_p, C.POINTER(occ_gbuffer), c_void_p, c_void_p]),
    "occ_tile_gbuffer": (c_int32, [c_void_p, C.POINTER(occ_gbuffer), c_void_p, c_void_p, c_void_p]),
    "occ_debug_bvh_host": (c_int32, [c_void_p, c_int64, c_void_p, c_int64, c_void_p, c_int64,
                                     C.POINTER(c_int64), C.POINTER(c_int32)]),
    "occ_trace_ao": (c_int32, [c_void_p, C.POINTER(occ_gbuffer), c_void_p, c_float, c_uint64,
                               c_uint32, C.POINTER(occ_occluders), c_void_p]),
    "occ_trace_shadow": (c_int32, [c_void_p, C.POINTER(occ_gbuffer), c_void_p,
                                   C.POINTER(occ_rect_light), c_uint64, c_uint32,
                                   C.POINTER(occ_occluders), c_void_p]),
    "occ_reuse_ao": (c_int32, [c_void_p, C.POINTER(occ_gbuffer), C.POINTER(occ_occluders),
                               C.POINTER(occ_pattern), c_int32, c_int32, c_void_p, c_void_p,
                               c_void_p]),
    "occ_reuse_shadow": (c_int32, [c_void_p, C.POINTER(occ_gbuffer), C.POINTER(occ_occluders),
                                   C.POINTER(occ_pattern), c_int32, c_int32, c_void_p, c_void_p,
                                   c_void_p]),
    "occ_trace_reuse_ao": (c_int32, [c_void_p, C.POINTER(occ_gbuffer), c_void_p, c_float,
                                     c_uint64, c_uint32, C.POINTER(occ_pattern), c_int32, c_int32,
                                     c_void_p, c_void_p, c_void_p]),
    "occ_trace_reuse_shadow": (c_int32, [c_void_p, C.POINTER(occ_gbuffer), c_void_p,
                                         C.POINTER(occ_rect_light), c_uint64, c_uint32,
                                         C.POINTER(occ_pattern), c_int32, c_int32, c_void_p,
                                         c_void_p, c_void_p]),
    "occ_frame_host": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p, c_int32,
                                 c_int32, c_float, C.POINTER(occ_rect_light), c_uint64, c_uint32,
                                 C.POINTER(occ_pattern), c_int32, c_int32, c_void_p, c_void_p]),
    "occ_frame_host_async": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p, c_int32,
                                       c_int32, c_float, C.POINTER(occ_rect_light), c_uint64,
                                       c_uint32, C.POINTER(occ_pattern), c_int32, c_int32,
                                       c_void_p, c_void_p]),
    "occ_frame_noalloc": (c_int32, [C.POINTER(occ_gbuffer), c_void_p, c_int32, c_float,
                                    C.POINTER(occ_rect_light), c_uint64, c_uint32,
                                    C.POINTER(occ_pattern), c_int32, c_int32, c_void_p, c_void_p,
                                    c_char_p, c_int32, c_void_p]),
    "occ_shadow_lights": (c_int32, [c_void_p, C.POINTER(occ_gbuffer), c_void_p,
                                    C.POINTER(occ_rect_light), c_void_p, c_int32, c_uint64,
                                    c_uint32, C.POINTER(occ_pattern), c_int32, c_int32,
                                    C.POINTER(occ_occluders), c_void_p, c_void_p, c_void_p]),
    "occ_frame_batch": (c_int32, [c_void_p, c_void_p, C.POINTER(occ_view), c_int32, c_void_p]),
    "occ_batch_capture": (c_int32, [c_void_p, c_void_p, C.POINTER(occ_view), c_int32,
                                    C.POINTER(c_void_p)]),
    "occ_batch_launch": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "occ_batch_free": (c_int32, [c_void_p, c_void_p]),
    "occ_set_tuning": (c_int32, [c_void_p, C.POINTER(occ_tuning)]),
    "occ_get_tuning": (c_int32, [c_void_p, C.POINTER(occ_tuning)]),
    "occ_sched_create": (c_int32, [C.POINTER(occ_sched_config), C.POINTER(c_void_p)]),
    "occ_sched_destroy": (c_int32, [c_void_p]),
    "occ_sched_submit": (c_int32, [c_void_p, c_uint64, c_int64, c_int64, c_int64]),
    "occ_sched_next": (c_int32, [c_void_p, c_int64, c_void_p, c_int32, C.POINTER(c_int32),
                                 C.POINTER(c_int32), c_void_p, c_int32, C.POINTER(c_int32)]),
    "occ_sched_complete": (c_int32, [c_void_p, c_int32]),
    "occ_sched_drain": (c_int32, [c_void_p, c_void_p, c_int32, C.POINTER(c_int32)]),
    "occ_sched_get_stats": (c_int32, [c_void_p, C.POINTER(occ_sched_stats)]),
    "occ_server_create": (c_int32, [c_void_p, c_void_p, C.POINTER(occ_server_config),
                                    C.POINTER(c_void_p)]),
    "occ_server_submit": (c_int32, [c_void_p, C.POINTER(occ_request), C.POINTER(c_uint64),
                                    c_char_p, c_int32]),
    "occ_server_poll": (c_int32, [c_void_p, C.POINTER(occ_result), c_int32, c_int64,
                                  C.POINTER(c_int32)]),
    "occ_server_get_stats": (c_int32, [c_void_p, C.POINTER(occ_server_stats)]),
    "occ_server_shutdown": (c_int32, [c_void_p, c_int32]),
    "occ_server_destroy": (c_int32, [c_void_p, c_int32]),
    "occ_debug_wait_timeout": (c_int32, [c_void_p, c_uint32, c_void_p]),
    "occ_debug_fp32_peak": (c_int32, [c_void_p, c_int32, c_int32, c_int32, c_void_p,
                                      C.POINTER(c_double), c_void_p]),
    "occ_debug_bvh_counters": (c_int32, [c_void_p, c_void_p, c_int32, C.POINTER(c_uint64)]),
    "occ_debug_stream_ceiling": (c_int32, [c_void_p, C.POINTER(occ_gbuffer), C.POINTER(occ_occluders),
                                           c_void_p, c_void_p]),
    "occ_debug_closest_hit": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_void_p,
                                        c_void_p, c_void_p]),
    "occ_debug_philox": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p]),
    "occ_debug_rays": (c_int32, [c_void_p, C.POINTER(occ_gbuffer), c_int32, c_float,
                                 C.POINTER(occ_rect_light), c_uint64, c_uint32, c_void_p,
                                 c_void_p]),
    "occ_debug_mis": (c_int32, [c_void_p, C.POINTER(occ_gbuffer), C.POINTER(occ_occluders),
                                C.POINTER(occ_pattern), c_int32, c_int32, c_void_p, c_void_p,
                                c_int32, c_void_p, c_void_p]),
}

_lock = threading.Lock()
_lib = None


def variant() -> str:
    return os.environ.get("OCC_LIB_VARIANT", "")


def library_path() -> str:
    return _lib_path(variant())


def load(build_if_missing: bool = True) -> C.CDLL:
    """Loads liboccreuse.so (building it first if allowed); raises if it is unavailable."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        var = variant()
        path = _lib_path(var)
        if not os.path.exists(path) or not _up_to_date(var):
            if not build_if_missing:
                raise RuntimeError(f"{os.path.basename(path)} is not built ({path}); run build()")
            _do_build(variant=var)
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib
