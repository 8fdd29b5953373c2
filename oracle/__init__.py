"""CPU oracle of the binned forward rasterizer (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's timed CPU
baseline load this package.  The library is plain C (``piko_oracle.c``),
built with gcc on first use; it shares no code with the CUDA path.  The
functions here marshal numpy arrays and return numpy results.

Functions without a pin against something other than this code: none of the
fixed-point conventions can be pinned to the paper, which is silent on them
(see the header of ``piko_oracle.c``); they are pinned to closed forms,
invariants and the separately written scanline rasterizer by the tests.
Near/far clipping (O16, ``set_clipping``) is a process-wide switch of the
library: set it around calls, not from concurrent threads.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "piko_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libpiko_oracle.so")
_lock = threading.Lock()
_lib = None

KEY_EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)
OK = 0
BAD_INDEX = 6


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no contraction, no fast-math)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-pthread", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        P = C.c_void_p
        i32, i64 = C.c_int, C.c_int64
        lib.oracle_vertex_stage.argtypes = [i32, i32, i32, P, P, P, P, P, P]
        lib.oracle_raster_brute.argtypes = [i32, i32, i32, P, i64, P, P, P, P]
        lib.oracle_keys_at.argtypes = [i32, i32, i32, P, i64, P, P, i64, P, P]
        lib.oracle_raster_bbox.argtypes = [i32, i32, i32, P, i64, P, P, P, i32]
        lib.oracle_raster_scanline.argtypes = [i32, i32, i32, P, i64, P, P, P]
        lib.oracle_half_from_double.argtypes = [C.c_double]
        lib.oracle_half_from_double.restype = C.c_uint16
        lib.oracle_double_from_half.argtypes = [C.c_uint16]
        lib.oracle_double_from_half.restype = C.c_double
        lib.oracle_shade.argtypes = [i32, i32, i32, P, i64, P, P, P, P, P, i32, i32, P, P, P, P]
        lib.oracle_light_pass.argtypes = [i32, i32, P, P, P, i32, P, P]
        lib.oracle_backward.argtypes = [i32, i32, i32, P, i64, P, P, P, P, P, i32, i32, P, P, P, P, P]
        lib.oracle_loss.argtypes = [i32, i32, i32, P, i64, P, P, P, P, P, i32, i32, P, P]
        lib.oracle_loss.restype = C.c_double
        lib.oracle_set_clipping.argtypes = [i32]
        lib.oracle_set_clipping.restype = None
        lib.oracle_get_clipping.argtypes = []
        lib.oracle_get_clipping.restype = i32
        lib.oracle_clip_count.argtypes = [i32, i32, i32, P, i64, P, P, P]
        _lib = lib
        return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _geom(scene, mvp=None):
    pos = np.ascontiguousarray(scene.pos, dtype=np.float32)
    tris = np.ascontiguousarray(scene.tris, dtype=np.int32)
    M = scene.mvp if mvp is None else mvp
    M = None if M is None else np.ascontiguousarray(M, dtype=np.float32).reshape(16)
    return pos, tris, M


def vertex_stage(scene, mvp=None):
    """O1-O5 per vertex: (X int32, Y int32, Z uint32, ok int32)."""
    lib = _load()
    pos, _, M = _geom(scene, mvp)
    V = pos.shape[0]
    X = np.zeros(V, np.int32)
    Y = np.zeros(V, np.int32)
    Z = np.zeros(V, np.uint32)
    ok = np.zeros(V, np.int32)
    lib.oracle_vertex_stage(scene.width, scene.height, V, _p(pos), _p(M), _p(X), _p(Y), _p(Z), _p(ok))
    return X, Y, Z, ok


def raster_brute(scene, mvp=None, with_count=False):
    """Every pixel against every triangle: key uint64 [H,W] (+ inside counts)."""
    lib = _load()
    pos, tris, M = _geom(scene, mvp)
    key = np.empty((scene.height, scene.width), np.uint64)
    cnt = np.empty((scene.height, scene.width), np.uint32) if with_count else None
    st = lib.oracle_raster_brute(scene.width, scene.height, pos.shape[0], _p(pos), tris.shape[0],
                                 _p(tris), _p(M), _p(key), _p(cnt))
    return (key, cnt, st) if with_count else (key, st)


def raster_bbox(scene, mvp=None, threads=1):
    """Bounding-box restricted evaluation of the same definition."""
    lib = _load()
    pos, tris, M = _geom(scene, mvp)
    key = np.empty((scene.height, scene.width), np.uint64)
    st = lib.oracle_raster_bbox(scene.width, scene.height, pos.shape[0], _p(pos), tris.shape[0],
                                _p(tris), _p(M), _p(key), int(threads))
    return key, st


def raster_scanline(scene, mvp=None):
    """The independently written scanline rasterizer."""
    lib = _load()
    pos, tris, M = _geom(scene, mvp)
    key = np.empty((scene.height, scene.width), np.uint64)
    st = lib.oracle_raster_scanline(scene.width, scene.height, pos.shape[0], _p(pos), tris.shape[0],
                                    _p(tris), _p(M), _p(key))
    return key, st


def keys_at(scene, pix_xy, mvp=None):
    """Brute-force keys at the listed pixels (int32 [N,2] of x, y)."""
    lib = _load()
    pos, tris, M = _geom(scene, mvp)
    pix = np.ascontiguousarray(pix_xy, dtype=np.int32).reshape(-1, 2)
    key = np.empty(pix.shape[0], np.uint64)
    st = lib.oracle_keys_at(scene.width, scene.height, pos.shape[0], _p(pos), tris.shape[0], _p(tris),
                            _p(M), pix.shape[0], _p(pix), _p(key))
    return key, st


def _d(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _flags(unclamped, perspective):
    return (1 if unclamped else 0) | (2 if perspective else 0)


def shade(scene, key, mvp=None, color=None, normal=None, light=None, mode=None, unclamped=False,
          perspective=False):
    """Float64 shading of the oracle's key buffer.  Returns rgba [H,W,4] float64
    for modes 0/1, or (normal_half, albedo_half) uint16 [H,W,4] for mode 2.
    color / normal / light default to the scene's, as float64.  perspective:
    perspective-correct barycentrics (O15) instead of screen-space ones."""
    lib = _load()
    pos, tris, M = _geom(scene, mvp)
    mode = scene.shade_mode if mode is None else mode
    col = _d(scene.color if color is None else color)
    nrm = _d(scene.normal if normal is None else normal)
    L = _d(scene.light_dir if light is None else light)
    if L is None:
        L = np.zeros(3)
    key = np.ascontiguousarray(key, dtype=np.uint64)
    H, W = scene.height, scene.width
    if mode == 2:
        gn = np.empty((H, W, 4), np.uint16)
        ga = np.empty((H, W, 4), np.uint16)
        lib.oracle_shade(W, H, pos.shape[0], _p(pos), tris.shape[0], _p(tris), _p(M), _p(col), _p(nrm),
                         _p(L), 2, _flags(unclamped, perspective), _p(key), None, _p(gn), _p(ga))
        return gn, ga
    rgba = np.empty((H, W, 4), np.float64)
    lib.oracle_shade(W, H, pos.shape[0], _p(pos), tris.shape[0], _p(tris), _p(M), _p(col), _p(nrm), _p(L),
                     int(mode), _flags(unclamped, perspective), _p(key), _p(rgba), None, None)
    return rgba


def light_pass(key, gnormal_u16, galbedo_u16, lights):
    """Float64 light pass over a G-buffer (binary16 given as uint16 bits)."""
    lib = _load()
    key = np.ascontiguousarray(key, dtype=np.uint64)
    H, W = key.shape
    gn = np.ascontiguousarray(gnormal_u16).view(np.uint16)
    ga = np.ascontiguousarray(galbedo_u16).view(np.uint16)
    lt = np.ascontiguousarray(lights, dtype=np.float32).reshape(-1, 4)
    rgba = np.empty((H, W, 4), np.float64)
    lib.oracle_light_pass(W, H, _p(key), _p(gn), _p(ga), lt.shape[0], _p(lt), _p(rgba))
    return rgba


def backward(scene, key, dl_drgba, mvp=None, color=None, normal=None, light=None, mode=None,
             unclamped=False, out=None, perspective=False):
    """Float64 analytic gradients (dcolor [V,3], dnormal [V,3], dlight [3]),
    accumulated into ``out`` when given."""
    lib = _load()
    pos, tris, M = _geom(scene, mvp)
    mode = scene.shade_mode if mode is None else mode
    col = _d(scene.color if color is None else color)
    nrm = _d(scene.normal if normal is None else normal)
    L = _d(scene.light_dir if light is None else light)
    if L is None:
        L = np.zeros(3)
    V = pos.shape[0]
    if out is None:
        out = (np.zeros((V, 3)), np.zeros((V, 3)), np.zeros(3))
    dc, dn, dl = out
    g = np.ascontiguousarray(dl_drgba, dtype=np.float64)
    key = np.ascontiguousarray(key, dtype=np.uint64)
    lib.oracle_backward(scene.width, scene.height, V, _p(pos), tris.shape[0], _p(tris), _p(M), _p(col),
                        _p(nrm), _p(L), int(mode), _flags(unclamped, perspective), _p(key), _p(g), _p(dc),
                        _p(dn), _p(dl))
    return dc, dn, dl


def loss(scene, key, target, mvp=None, color=None, normal=None, light=None, mode=None,
         unclamped=False, perspective=False) -> float:
    """sum (rgb - target)^2 over pixels and RGB, float64, visibility fixed."""
    lib = _load()
    pos, tris, M = _geom(scene, mvp)
    mode = scene.shade_mode if mode is None else mode
    col = _d(scene.color if color is None else color)
    nrm = _d(scene.normal if normal is None else normal)
    L = _d(scene.light_dir if light is None else light)
    if L is None:
        L = np.zeros(3)
    key = np.ascontiguousarray(key, dtype=np.uint64)
    tgt = np.ascontiguousarray(target, dtype=np.float32)
    return float(lib.oracle_loss(scene.width, scene.height, pos.shape[0], _p(pos), tris.shape[0], _p(tris),
                                 _p(M), _p(col), _p(nrm), _p(L), int(mode), _flags(unclamped, perspective),
                                 _p(key), _p(tgt)))


def half_from_double(x: float) -> int:
    return int(_load().oracle_half_from_double(float(x)))


def double_from_half(h: int) -> float:
    return float(_load().oracle_double_from_half(int(h)))


def set_clipping(on: bool) -> None:
    """O16: near/far clipping instead of the culls of O2/O3 for every later
    call (a process-wide switch of the library; off by default)."""
    _load().oracle_set_clipping(1 if on else 0)


def get_clipping() -> bool:
    return bool(_load().oracle_get_clipping())


class clipping:
    """Context manager: O16 clipping on (or off) inside the block."""

    def __init__(self, on: bool = True):
        self.on = on

    def __enter__(self):
        self.prev = get_clipping()
        set_clipping(self.on)
        return self

    def __exit__(self, *exc):
        set_clipping(self.prev)
        return False


def clip_count(scene, mvp=None) -> int:
    """Number of sub-triangles the clipping step (O16) makes of the scene."""
    lib = _load()
    pos, tris, M = _geom(scene, mvp)
    n = C.c_int64(0)
    lib.oracle_clip_count(scene.width, scene.height, pos.shape[0], _p(pos), tris.shape[0], _p(tris), _p(M),
                          C.byref(n))
    return int(n.value)
