"""ctypes binding of libtets.so (include/tets.h): structures and entry points
with the same names.  Argument marshalling only."""

from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtets.so")

TTS_OK = 0
TTS_ERR_ARG = 1
TTS_ERR_WORKSPACE = 2
TTS_ERR_OVERFLOW = 3
TTS_ERR_CUDA = 4
TTS_ERR_TIMEOUT = 5
TTS_ERR_BAD_INDEX = 6

TTS_STATUS_BAD_INDEX = 1
TTS_STATUS_SURV_OVERFLOW = 2
TTS_STATUS_KEY_OVERFLOW = 4
TTS_STATUS_TIMEOUT = 8

TTS_FLAG_PURE = 1
TTS_FLAG_ACCUM_GRAD = 2
TTS_FLAG_FORWARD_ONLY = 4
TTS_FLAG_NORMALS = 8
TTS_FLAG_HULL = 16
TTS_FLAG_COUNT = 32

TTS_MAX_SCENES = 64
TTS_MAX_VIEWS = 128
TTS_SORT_NOALLOC_MAX_KEYS = 1 << 20


class tts_camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("znear", ctypes.c_float), ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class tts_params(ctypes.Structure):
    _fields_ = [("s", ctypes.c_float), ("prefilter_thresh", ctypes.c_float),
                ("alpha_skip", ctypes.c_float), ("alpha_cap", ctypes.c_float),
                ("t_eps", ctypes.c_float), ("tile", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("resort_window", ctypes.c_int32), ("blend_segment", ctypes.c_int32),
                ("blend_warps", ctypes.c_int32), ("frag_cap", ctypes.c_int32)]


class tts_scene(ctypes.Structure):
    _fields_ = [("V", ctypes.c_void_p), ("T", ctypes.c_void_p), ("f", ctypes.c_void_p),
                ("rgb", ctypes.c_void_p), ("N", ctypes.c_int64), ("K", ctypes.c_int64),
                ("surv_capacity", ctypes.c_int64)]


class tts_view(ctypes.Structure):
    _fields_ = [("cam", tts_camera), ("scene", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class tts_batch(ctypes.Structure):
    _fields_ = [("scenes", ctypes.POINTER(tts_scene)), ("n_scenes", ctypes.c_int32),
                ("views", ctypes.POINTER(tts_view)), ("n_views", ctypes.c_int32),
                ("params", tts_params), ("key_capacity", ctypes.c_int64),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t)]


class tts_outputs(ctypes.Structure):
    _fields_ = [("image", ctypes.c_void_p), ("alpha", ctypes.c_void_p), ("depth", ctypes.c_void_p),
                ("normal", ctypes.c_void_p)]


class tts_upstream(ctypes.Structure):
    _fields_ = [("dimage", ctypes.c_void_p), ("dalpha", ctypes.c_void_p),
                ("ddepth", ctypes.c_void_p), ("dnormal", ctypes.c_void_p)]


class tts_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_uint32), ("n_scenes", ctypes.c_int32),
                ("n_keys", ctypes.c_int64), ("n_surv", ctypes.c_int64 * TTS_MAX_SCENES),
                ("sort_bits", ctypes.c_int32), ("long_lists", ctypes.c_int32),
                ("blend_units", ctypes.c_int32), ("reserved", ctypes.c_int32)]


ENTRY_POINTS = ("tts_workspace_size", "tts_workspace_init", "tts_prepare_scene",
                "tts_survivor_bounds", "tts_fit_grid", "tts_render_fwd",
                "tts_render_bwd", "tts_render_fwd_ex", "tts_render_bwd_ex", "tts_bin_views",
                "tts_blend_fwd", "tts_blend_bwd", "tts_blend_fwd_ex", "tts_blend_bwd_ex",
                "tts_scatter_bwd", "tts_launch_count", "tts_debug_pixels", "tts_debug_frag_lists",
                "tts_debug_walk_counts",
                "tts_get_info",
                "tts_debug_lists", "tts_debug_records", "tts_sort_pairs_noalloc",
                "tts_sort_pairs_scratch_size", "tts_sort_pairs",
                "tts_tet_edges_workspace_size", "tts_tet_edges", "tts_regularizers_workspace_size",
                "tts_regularizers", "tts_marching_tets_workspace_size", "tts_marching_tets",
                "tts_geometry_status", "tts_debug_scan_wait", "tts_debug_kernel_events",
                "tts_debug_kernel_events_used",
                "tts_error_string", "tts_version")

_lib = None


class TetsError(RuntimeError):
    pass


def load():
    """Loads libtets.so from the package directory.  Raises when it has not
    been built: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise TetsError(f"{LIB_PATH} is missing: build it with "
                        "`python -m paper_2406_01579_b300.build`")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    B = ctypes.POINTER(tts_batch)
    L.tts_workspace_size.argtypes = [B, ctypes.POINTER(ctypes.c_size_t)]
    L.tts_workspace_init.argtypes = [B, P]
    L.tts_prepare_scene.argtypes = [B, P]
    L.tts_render_fwd.argtypes = [B, P, P, P, P]
    L.tts_render_bwd.argtypes = [B, P, P, P, P, P, P, P]
    O = ctypes.POINTER(tts_outputs)
    U = ctypes.POINTER(tts_upstream)
    L.tts_render_fwd_ex.argtypes = [B, O, P]
    L.tts_render_bwd_ex.argtypes = [B, U, P, P, P, P]
    L.tts_blend_fwd_ex.argtypes = [B, O, P]
    L.tts_blend_bwd_ex.argtypes = [B, U, P]
    L.tts_survivor_bounds.argtypes = [B, P, P]
    F3 = ctypes.c_float * 3
    L.tts_fit_grid.argtypes = [P, ctypes.c_int64, F3, F3, P, ctypes.c_float, P, P]
    L.tts_bin_views.argtypes = [B, P]
    L.tts_blend_fwd.argtypes = [B, P, P, P, P]
    L.tts_blend_bwd.argtypes = [B, P, P, P, P]
    L.tts_scatter_bwd.argtypes = [B, P, P, P, P]
    L.tts_launch_count.argtypes = []
    L.tts_debug_pixels.argtypes = [B, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), P]
    L.tts_debug_frag_lists.argtypes = [B, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P),
                                       ctypes.POINTER(ctypes.c_int32), P]
    L.tts_debug_walk_counts.argtypes = [B, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int32, P]
    L.tts_get_info.argtypes = [B, ctypes.POINTER(tts_info), P]
    L.tts_debug_lists.argtypes = [B, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P),
                                  ctypes.POINTER(P), ctypes.POINTER(ctypes.c_uint32),
                                  ctypes.POINTER(ctypes.c_int32), P]
    L.tts_debug_records.argtypes = [B, ctypes.POINTER(P), P]
    L.tts_sort_pairs_noalloc.argtypes = [P, P, P, P, ctypes.c_int64, ctypes.c_int32, P]
    L.tts_sort_pairs_scratch_size.argtypes = [ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)]
    L.tts_sort_pairs.argtypes = [P, P, P, P, ctypes.c_int64, ctypes.c_int32, P, ctypes.c_size_t, P]
    i64 = ctypes.c_int64
    L.tts_tet_edges_workspace_size.argtypes = [i64, i64, ctypes.POINTER(ctypes.c_size_t)]
    L.tts_tet_edges.argtypes = [P, i64, i64, P, i64, P, P, ctypes.c_size_t, P]
    L.tts_regularizers_workspace_size.argtypes = [i64, ctypes.POINTER(ctypes.c_size_t)]
    L.tts_regularizers.argtypes = [P, P, P, i64, i64, P, i64, ctypes.c_float, ctypes.c_float, P,
                                   P, P, ctypes.c_int32, P, ctypes.c_size_t, P]
    L.tts_marching_tets_workspace_size.argtypes = [i64, i64, ctypes.POINTER(ctypes.c_size_t)]
    L.tts_marching_tets.argtypes = [P, P, P, i64, i64, P, i64, P, P, i64, P, i64, P, P,
                                    ctypes.c_size_t, P]
    L.tts_geometry_status.argtypes = [P, ctypes.POINTER(ctypes.c_uint32), P]
    L.tts_debug_scan_wait.argtypes = [ctypes.c_int64, ctypes.c_int32]
    L.tts_debug_kernel_events.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32]
    L.tts_debug_kernel_events_used.argtypes = [ctypes.POINTER(ctypes.c_char_p), ctypes.c_int32]
    L.tts_error_string.argtypes = [ctypes.c_int]
    L.tts_error_string.restype = ctypes.c_char_p
    L.tts_version.argtypes = []
    L.tts_version.restype = ctypes.c_char_p
    for name in ENTRY_POINTS:
        if name not in ("tts_error_string", "tts_version"):
            getattr(L, name).restype = ctypes.c_int
    L.tts_launch_count.restype = ctypes.c_int64
    L.tts_debug_kernel_events_used.restype = ctypes.c_int32
    _lib = L
    return L


def check(rc: int, what: str = ""):
    if rc != TTS_OK:
        msg = load().tts_error_string(rc).decode()
        raise TetsError(f"{what}: {msg} (code {rc})")
