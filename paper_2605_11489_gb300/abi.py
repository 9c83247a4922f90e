"""ctypes binding of include/gsr.h (argument marshalling only).

Every computation happens inside libgsr.so. Loading fails loudly when the
library has not been built (run ``__graft_entry__.build()`` or
``python -m paper_2605_11489_gb300.build``): there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
# GSR_DEBUG=1 loads the GSR_DEBUG build (build.build(debug=True)), whose device index guards
# report kErrBounds as GS_ERR_INTERNAL
LIB_PATH = os.path.join(HERE, "libgsr_debug.so" if os.environ.get("GSR_DEBUG") == "1" else "libgsr.so")

GS_OK = 0
GS_NOT_READY = 1
GS_ERR_INVALID_ARG = -1
GS_ERR_OOM = -2
GS_ERR_CUDA = -3
GS_ERR_TIMEOUT = -4
GS_ERR_CAPACITY = -5
GS_ERR_CANCELLED = -6
GS_ERR_INTERNAL = -7
GS_EMIT_BWD_STATE = 1
GS_TIME_STAGES = 2
GS_TIME_COMPOSITE = 8
GS_COUNT_PAIRS = 4
STAGES = ("project", "scan", "compact", "depth_sort", "duplicate", "tile_sort", "ranges", "composite")

STATUS_NAMES = {0: "GS_OK", 1: "GS_NOT_READY", -1: "GS_ERR_INVALID_ARG", -2: "GS_ERR_OOM", -3: "GS_ERR_CUDA",
                -4: "GS_ERR_TIMEOUT", -5: "GS_ERR_CAPACITY", -6: "GS_ERR_CANCELLED",
                -7: "GS_ERR_INTERNAL"}

# every entry point declared in include/gsr.h
ENTRY_POINTS = (
    "gs_context_create", "gs_context_destroy", "gs_render_forward", "gs_render_forward_to_host",
    "gs_render_backward", "gs_state_view_get", "gs_context_stats", "gs_context_check", "gs_context_debug_waits",
    "gs_state_free", "gs_graph_create",
    "gs_graph_render", "gs_graph_check", "gs_graph_stats", "gs_graph_destroy", "gs_frame_stream_create",
    "gs_frame_stream_submit", "gs_frame_stream_join", "gs_frame_stream_release", "gs_frame_stream_wait",
    "gs_frame_stream_synchronize", "gs_frame_stream_stats", "gs_frame_stream_destroy",
    "gs_autotune", "gs_server_create", "gs_server_load_scene",
    "gs_server_submit", "gs_server_poll", "gs_server_cancel", "gs_server_drain", "gs_server_destroy",
    "gs_sort_pairs_static", "gs_warp", "gs_gai_upsample", "gs_last_error", "gs_version",
)


class GsScene(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_pad", C.c_int64), ("sh_degree", C.c_int32), ("_reserved", C.c_int32),
                ("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p)]


class GsCamera(C.Structure):
    _fields_ = [("viewmat", C.c_float * 12), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float),
                ("cy", C.c_float), ("near_plane", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class GsRenderOpts(C.Structure):
    _fields_ = [("tile", C.c_int32), ("batch", C.c_int32), ("bg", C.c_float * 3), ("flags", C.c_uint32),
                ("chunk", C.c_int32), ("head", C.c_int32)]


class GsOutputs(C.Structure):
    _fields_ = [("rgb", C.c_void_p), ("dcdx", C.c_void_p), ("dcdy", C.c_void_p), ("depth", C.c_void_p),
                ("alpha", C.c_void_p), ("normal", C.c_void_p), ("nv", C.c_void_p),
                ("depth_isect", C.c_void_p)]


class GsSceneGrads(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p)]


class GsStateView(C.Structure):
    _fields_ = [("n_instances", C.c_int64), ("n_visible", C.c_int64), ("n_tiles", C.c_int32),
                ("tiles_x", C.c_int32), ("tiles_y", C.c_int32), ("tile", C.c_int32),
                ("keys", C.c_void_p), ("vals", C.c_void_p), ("ranges", C.c_void_p), ("ntiles", C.c_void_p),
                ("records", C.c_void_p), ("final_T", C.c_void_p), ("n_contrib", C.c_void_p)]


class GsFrameStats(C.Structure):
    _fields_ = [("frames", C.c_int64), ("instances_total", C.c_int64), ("visible_total", C.c_int64),
                ("instances_max", C.c_int64), ("stage_ms", C.c_double * len(STAGES)), ("timed_frames", C.c_int64),
                ("pairs_evaluated", C.c_int64), ("pairs_blended", C.c_int64)]


class GsWarpInput(C.Structure):
    _fields_ = [("depth", C.c_void_p), ("alpha", C.c_void_p), ("alpha_min", C.c_float), ("channels", C.c_int32),
                ("planes", C.c_void_p), ("grad_channels", C.c_int32), ("dcdx", C.c_void_p), ("dcdy", C.c_void_p)]


class GsWarpOutput(C.Structure):
    _fields_ = [("motion", C.c_void_p), ("index", C.c_void_p), ("z", C.c_void_p), ("planes", C.c_void_p),
                ("dcdx", C.c_void_p), ("dcdy", C.c_void_p)]


class GsGaiWeights(C.Structure):
    _fields_ = [("scale", C.c_int32), ("features", C.c_int32), ("wc", C.c_void_p), ("bc", C.c_void_p),
                ("wt", C.c_void_p), ("bt", C.c_void_p)]


class GsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lock = threading.Lock()
_lib = None


def _declare(L):
    P, I32, I64, U64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
    st = C.c_int
    sig = {
        "gs_context_create": [C.c_int, C.POINTER(P)],
        "gs_context_destroy": [P],
        "gs_render_forward": [P, C.POINTER(GsScene), C.POINTER(GsCamera), C.POINTER(GsRenderOpts),
                              C.POINTER(GsOutputs), C.POINTER(P), P],
        "gs_render_forward_to_host": [P, C.POINTER(GsScene), C.POINTER(GsCamera), C.POINTER(GsRenderOpts),
                                      C.POINTER(GsOutputs), P],
        "gs_render_backward": [P, P, C.POINTER(GsScene), C.POINTER(GsOutputs), C.POINTER(GsSceneGrads), P],
        "gs_state_view_get": [P, C.POINTER(GsStateView)],
        "gs_state_free": [P],
        "gs_graph_create": [P, C.POINTER(GsScene), C.POINTER(GsCamera), C.POINTER(GsRenderOpts),
                            C.POINTER(GsOutputs), I64, P, C.POINTER(P)],
        "gs_graph_render": [P, C.POINTER(GsCamera), P],
        "gs_graph_check": [P, P, C.POINTER(I64)],
        "gs_graph_destroy": [P],
        "gs_graph_stats": [P, P, C.c_int, C.POINTER(GsFrameStats)],
        "gs_frame_stream_create": [P, C.POINTER(GsScene), C.POINTER(GsCamera), C.POINTER(GsRenderOpts),
                                   C.POINTER(GsOutputs), I32, I64, C.POINTER(P)],
        "gs_frame_stream_submit": [P, C.POINTER(GsCamera), C.POINTER(GsOutputs), C.POINTER(I64)],
        "gs_frame_stream_join": [P, I64, P],
        "gs_frame_stream_release": [P, I64, P],
        "gs_frame_stream_wait": [P, I64],
        "gs_frame_stream_synchronize": [P],
        "gs_frame_stream_stats": [P, I32, C.c_int, C.POINTER(GsFrameStats)],
        "gs_frame_stream_destroy": [P],
        "gs_context_stats": [P, P, C.c_int, C.POINTER(GsFrameStats)],
        "gs_context_check": [P, P],
        "gs_context_debug_waits": [P, I32],
        "gs_autotune": [P, C.POINTER(GsScene), C.POINTER(GsCamera), C.POINTER(GsOutputs), C.c_int, P,
                        C.POINTER(I32), C.POINTER(I32), C.POINTER(I32), C.POINTER(C.c_float)],
        "gs_server_create": [C.c_int, C.c_size_t, C.c_int, C.POINTER(P)],
        "gs_server_load_scene": [P, C.POINTER(GsScene), C.POINTER(I32)],
        "gs_server_submit": [P, I32, C.POINTER(GsCamera), C.POINTER(GsRenderOpts), C.POINTER(GsOutputs),
                             C.POINTER(U64)],
        "gs_server_poll": [P, U64, C.POINTER(C.c_double)],
        "gs_server_cancel": [P, U64],
        "gs_server_drain": [P],
        "gs_server_destroy": [P],
        "gs_sort_pairs_static": [P, P, P, P, I64, I32, P, P],
        "gs_warp": [P, C.POINTER(GsCamera), C.POINTER(GsCamera), C.POINTER(GsWarpInput), C.POINTER(GsWarpOutput),
                    P],
        "gs_gai_upsample": [C.POINTER(GsGaiWeights), P, P, P, I32, I32, I32, P, P],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = st
    L.gs_last_error.restype = C.c_char_p
    L.gs_last_error.argtypes = []
    L.gs_version.restype = C.c_char_p
    L.gs_version.argtypes = []


def lib(path: str | None = None):
    """Load libgsr.so (raises if it is missing: the render path has no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError("libgsr.so not built (%s); run __graft_entry__.build()" % p)
            L = C.CDLL(p)
            _declare(L)
            _lib = L
    return _lib


def check(status: int) -> int:
    if status < 0:
        msg = lib().gs_last_error()
        raise GsError(status, msg.decode() if msg else "")
    return status


def last_error() -> str:
    m = lib().gs_last_error()
    return m.decode() if m else ""
