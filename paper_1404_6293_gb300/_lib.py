"""ctypes view of the C ABI in include/piko_raster.h (argument marshalling only).

The shared library is built in-tree by ``paper_1404_6293_gb300.build``.  If
it is missing and cannot be built, loading raises: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

PIKO_OK = 0
PIKO_ERR_INVALID_ARG = 1
PIKO_ERR_CUDA = 2
PIKO_ERR_OOM = 3
PIKO_ERR_OVERFLOW = 4
PIKO_ERR_TIMEOUT = 5
PIKO_ERR_BAD_INDEX = 6

PIKO_SCHED_STATIC = 0
PIKO_SCHED_DYNAMIC = 1
PIKO_SCHED_HARDWARE = 2
PIKO_SCHED_FUSED = 3
PIKO_SCHED_UNFUSED = 4

PIKO_SHADE_GOURAUD = 0
PIKO_SHADE_LAMBERT = 1
PIKO_SHADE_GBUFFER = 2

PIKO_OPT_THREADS_PER_TILE = 1
PIKO_OPT_UNCLAMPED = 2
PIKO_OPT_CHECK_CAPACITY = 3
PIKO_OPT_SCHEDULE = 4
PIKO_OPT_SMALL_TRI_PIXELS = 5
PIKO_OPT_STATS = 6
PIKO_OPT_BATCH_LAUNCH = 7
PIKO_OPT_PERSPECTIVE = 8
PIKO_OPT_WAIT_BUDGET = 9
PIKO_OPT_TEST_WITHHOLD = 10
PIKO_OPT_CLIP = 11
PIKO_OPT_EXACT_BINS = 12
PIKO_NUM_STAGE_EVENTS = 6

ERROR_NAMES = {
    PIKO_OK: "ok", PIKO_ERR_INVALID_ARG: "invalid argument", PIKO_ERR_CUDA: "CUDA error",
    PIKO_ERR_OOM: "out of memory", PIKO_ERR_OVERFLOW: "bin-list overflow",
    PIKO_ERR_TIMEOUT: "device wait timed out", PIKO_ERR_BAD_INDEX: "triangle index out of range",
}


class PikoScene(C.Structure):
    _fields_ = [
        ("width", C.c_int32), ("height", C.c_int32),
        ("num_vertices", C.c_int32), ("num_triangles", C.c_int32),
        ("pos", C.c_void_p), ("tris", C.c_void_p), ("color", C.c_void_p), ("normal", C.c_void_p),
        ("mvp", C.c_void_p), ("light_dir", C.c_void_p),
        ("shade_mode", C.c_int32), ("reserved", C.c_int32),
    ]


class PikoFramebuffer(C.Structure):
    _fields_ = [("key", C.c_void_p), ("rgba", C.c_void_p), ("gbuf_normal", C.c_void_p),
                ("gbuf_albedo", C.c_void_p)]


_lock = threading.Lock()
_lib = None


def _declare(lib):
    P = C.c_void_p
    i32, i64 = C.c_int, C.c_int64
    lib.piko_raster_create.argtypes = [i32, i32, i32, i32, i32]
    lib.piko_raster_create.restype = P
    lib.piko_raster_destroy.argtypes = [P]
    lib.piko_raster_destroy.restype = None
    lib.piko_raster_forward.argtypes = [P, C.POINTER(PikoScene), C.POINTER(PikoFramebuffer), P]
    lib.piko_raster_forward_host.argtypes = [P, C.POINTER(PikoScene), C.POINTER(PikoFramebuffer), P]
    lib.piko_raster_backward.argtypes = [P, C.POINTER(PikoScene), C.POINTER(PikoFramebuffer), P, P, P, P, P]
    lib.piko_raster_deferred_light.argtypes = [P, C.POINTER(PikoFramebuffer), P, i32, P, P]
    lib.piko_raster_reserve.argtypes = [P, i64, i64, i64]
    lib.piko_raster_set_option.argtypes = [P, i32, i32]
    lib.piko_raster_status.argtypes = [P, C.POINTER(C.c_int64)]
    lib.piko_raster_last_error.argtypes = [P]
    lib.piko_raster_last_error.restype = C.c_char_p
    lib.piko_raster_version.argtypes = []
    lib.piko_raster_set_stage_events.argtypes = [P, C.POINTER(C.c_void_p), i32]
    lib.piko_raster_stats.argtypes = [P, C.POINTER(C.c_int64)]
    for name in ("piko_raster_forward", "piko_raster_forward_host", "piko_raster_backward", "piko_raster_deferred_light",
                 "piko_raster_reserve", "piko_raster_set_option", "piko_raster_status",
                 "piko_raster_version", "piko_raster_set_stage_events", "piko_raster_stats"):
        getattr(lib, name).restype = i32
    lib.piko_raster_forward_batch.argtypes = [P, C.POINTER(PikoScene), i32, C.POINTER(PikoFramebuffer), P, P, P]
    lib.piko_raster_forward_batch.restype = i32
    lib.piko_raster_backward_batch.argtypes = [P, C.POINTER(PikoScene), i32, C.POINTER(PikoFramebuffer), P, P, P, P, P]
    lib.piko_raster_backward_batch.restype = i32
    return lib


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libpiko_raster.so, building it first if it is missing or stale."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and not _build.up_to_date():
            _build.build_library()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"{_build.LIB} is missing: build it with `python -m paper_1404_6293_gb300.build`")
        _lib = _declare(C.CDLL(_build.LIB))
        return _lib
