"""Python API of the GB300 binned rasterizer.

A thin wrapper over the C ABI (include/piko_raster.h): tensors supply device
memory and the current CUDA stream; every step of the pipeline runs in the
library's kernels.  There is no CPU path: without a CUDA device or the built
library, construction raises.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import _lib as L

KEY_EMPTY = 0xFFFFFFFFFFFFFFFF
_SCHEDULES = {"static": L.PIKO_SCHED_STATIC, "dynamic": L.PIKO_SCHED_DYNAMIC, "hardware": L.PIKO_SCHED_HARDWARE,
              "fused": L.PIKO_SCHED_FUSED, "unfused": L.PIKO_SCHED_UNFUSED}


class PikoError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{L.ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


@dataclass
class DeviceScene:
    """A scene resident on the GPU (tensors owned by Python)."""

    width: int
    height: int
    pos: torch.Tensor                      # float32 [V,4]
    tris: torch.Tensor                     # int32 [T,3]
    color: Optional[torch.Tensor] = None   # float32 [V,3]
    normal: Optional[torch.Tensor] = None  # float32 [V,3]
    mvp: Optional[torch.Tensor] = None     # float32 [16]
    light_dir: Optional[torch.Tensor] = None  # float32 [3]
    shade_mode: int = L.PIKO_SHADE_GOURAUD

    @staticmethod
    def from_host(scene, device="cuda", mvp=None) -> "DeviceScene":
        """Copies a host scene (numpy arrays, see scenes.Scene) to the device."""
        def t(a, dt):
            if a is None:
                return None
            return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(device)

        m = scene.mvp if mvp is None else mvp
        return DeviceScene(scene.width, scene.height, t(scene.pos, np.float32).reshape(-1, 4),
                           t(scene.tris, np.int32).reshape(-1, 3), t(scene.color, np.float32),
                           t(scene.normal, np.float32), None if m is None else t(m, np.float32).reshape(16),
                           t(scene.light_dir, np.float32), int(scene.shade_mode))

    @property
    def num_vertices(self) -> int:
        return int(self.pos.shape[0])

    @property
    def num_triangles(self) -> int:
        return int(self.tris.shape[0])

    def c_struct(self) -> L.PikoScene:
        for name in ("pos", "tris", "color", "normal", "mvp", "light_dir"):
            v = getattr(self, name)
            if v is not None and (not v.is_cuda or not v.is_contiguous()):
                raise ValueError(f"{name} must be a contiguous CUDA tensor")
        if self.pos.dtype != torch.float32 or self.tris.dtype != torch.int32:
            raise TypeError("pos must be float32 and tris int32")
        s = L.PikoScene()
        s.width, s.height = self.width, self.height
        s.num_vertices, s.num_triangles = self.num_vertices, self.num_triangles
        s.pos, s.tris = self.pos.data_ptr(), self.tris.data_ptr()
        s.color = None if self.color is None else self.color.data_ptr()
        s.normal = None if self.normal is None else self.normal.data_ptr()
        s.mvp = None if self.mvp is None else self.mvp.data_ptr()
        s.light_dir = None if self.light_dir is None else self.light_dir.data_ptr()
        s.shade_mode = self.shade_mode
        s.reserved = 0
        return s


@dataclass
class HostScene:
    """A scene in host memory (CPU tensors, pinned for asynchronous copies),
    for Rasterizer.forward_host: the library copies it to the device."""

    width: int
    height: int
    pos: torch.Tensor                      # float32 [V,4]
    tris: torch.Tensor                     # int32 [T,3]
    color: Optional[torch.Tensor] = None   # float32 [V,3]
    normal: Optional[torch.Tensor] = None  # float32 [V,3]
    mvp: Optional[torch.Tensor] = None     # float32 [16]
    light_dir: Optional[torch.Tensor] = None  # float32 [3]
    shade_mode: int = L.PIKO_SHADE_GOURAUD

    @staticmethod
    def from_host(scene, pin=True, mvp=None) -> "HostScene":
        """Wraps a host scene (numpy arrays, see scenes.Scene) in CPU tensors."""
        def t(a, dt):
            if a is None:
                return None
            x = torch.from_numpy(np.ascontiguousarray(a, dtype=dt).copy())
            return x.pin_memory() if pin else x

        m = scene.mvp if mvp is None else mvp
        return HostScene(scene.width, scene.height, t(scene.pos, np.float32).reshape(-1, 4),
                         t(scene.tris, np.int32).reshape(-1, 3), t(scene.color, np.float32),
                         t(scene.normal, np.float32), None if m is None else t(m, np.float32).reshape(16),
                         t(scene.light_dir, np.float32), int(scene.shade_mode))

    def c_struct(self) -> L.PikoScene:
        for name in ("pos", "tris", "color", "normal", "mvp", "light_dir"):
            v = getattr(self, name)
            if v is not None and (v.is_cuda or not v.is_contiguous()):
                raise ValueError(f"{name} must be a contiguous CPU tensor")
        if self.pos.dtype != torch.float32 or self.tris.dtype != torch.int32:
            raise TypeError("pos must be float32 and tris int32")
        s = L.PikoScene()
        s.width, s.height = self.width, self.height
        s.num_vertices, s.num_triangles = int(self.pos.shape[0]), int(self.tris.shape[0])
        s.pos, s.tris = self.pos.data_ptr(), self.tris.data_ptr()
        s.color = None if self.color is None else self.color.data_ptr()
        s.normal = None if self.normal is None else self.normal.data_ptr()
        s.mvp = None if self.mvp is None else self.mvp.data_ptr()
        s.light_dir = None if self.light_dir is None else self.light_dir.data_ptr()
        s.shade_mode = self.shade_mode
        s.reserved = 0
        return s


@dataclass
class Framebuffer:
    key: torch.Tensor                     # int64 [H,W] holding the uint64 keys
    rgba: Optional[torch.Tensor] = None   # float32 [H,W,4]
    gbuf_normal: Optional[torch.Tensor] = None  # float16 [H,W,4]
    gbuf_albedo: Optional[torch.Tensor] = None  # float16 [H,W,4]

    @staticmethod
    def allocate(width, height, mode=L.PIKO_SHADE_GOURAUD, device="cuda", rgba=True) -> "Framebuffer":
        key = torch.empty((height, width), dtype=torch.int64, device=device)
        if mode == L.PIKO_SHADE_GBUFFER:
            return Framebuffer(key, None, torch.empty((height, width, 4), dtype=torch.float16, device=device),
                               torch.empty((height, width, 4), dtype=torch.float16, device=device))
        return Framebuffer(key, torch.empty((height, width, 4), dtype=torch.float32, device=device) if rgba else None)

    def c_struct(self) -> L.PikoFramebuffer:
        f = L.PikoFramebuffer()
        f.key = self.key.data_ptr()
        f.rgba = None if self.rgba is None else self.rgba.data_ptr()
        f.gbuf_normal = None if self.gbuf_normal is None else self.gbuf_normal.data_ptr()
        f.gbuf_albedo = None if self.gbuf_albedo is None else self.gbuf_albedo.data_ptr()
        return f

    def key_numpy(self) -> np.ndarray:
        return self.key.cpu().numpy().view(np.uint64)


class Rasterizer:
    """One rasterizer handle: framebuffer size, bin size and tile schedule.

    schedule: "static" (DirectMap), "dynamic" (LoadBalance), "hardware"
    (one CTA per tile), or one of the other pipeline mappings: "fused" (no
    tiling, global depth buffer) and "unfused" (one kernel per stage)."""

    def __init__(self, width: int, height: int, bin_w: int = 16, bin_h: int = 16, schedule="static"):
        if not torch.cuda.is_available():
            raise RuntimeError("the rasterizer needs a CUDA device; there is no CPU path")
        self.lib = L.load()
        torch.cuda.current_device()  # makes sure torch's context is the current one
        sched = _SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule)
        h = self.lib.piko_raster_create(int(width), int(height), int(bin_w), int(bin_h), sched)
        if not h:
            raise PikoError(L.PIKO_ERR_INVALID_ARG,
                            f"piko_raster_create({width}, {height}, {bin_w}, {bin_h}, {schedule}) failed")
        self._h = C.c_void_p(h)
        self.width, self.height, self.bin_w, self.bin_h, self.schedule = width, height, bin_w, bin_h, sched

    # -------------------------------------------------------------- utils
    def _check(self, code: int):
        if code != L.PIKO_OK:
            raise PikoError(code, self.lib.piko_raster_last_error(self._h).decode())

    @staticmethod
    def _stream(stream) -> C.c_void_p:
        s = torch.cuda.current_stream() if stream is None else stream
        return C.c_void_p(s.cuda_stream)

    def close(self):
        if getattr(self, "_h", None):
            self.lib.piko_raster_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, key: int, value: int):
        self._check(self.lib.piko_raster_set_option(self._h, int(key), int(value)))

    def reserve(self, max_vertices: int, max_triangles: int, max_bin_entries: int):
        self._check(self.lib.piko_raster_reserve(self._h, int(max_vertices), int(max_triangles),
                                                 int(max_bin_entries)))

    def set_stage_events(self, events):
        """Records the given torch.cuda.Event objects (PIKO_NUM_STAGE_EVENTS of
        them, already created) at the stage boundaries of the next forward;
        None stops the recording."""
        if events is None:
            self._check(self.lib.piko_raster_set_stage_events(self._h, None, 0))
            return
        arr = (C.c_void_p * L.PIKO_NUM_STAGE_EVENTS)(*[C.c_void_p(e.cuda_event) for e in events])
        self._check(self.lib.piko_raster_set_stage_events(self._h, arr, L.PIKO_NUM_STAGE_EVENTS))

    def stats(self):
        """Work counted by the last forward run with PIKO_OPT_STATS = 1."""
        out = (C.c_int64 * 5)()
        self._check(self.lib.piko_raster_stats(self._h, out))
        return {"bin_entries": out[0], "samples_tested": out[1], "fragments": out[2], "shaded": out[3],
                "binned_triangles": out[4]}

    def status(self):
        """(code, needed bin entries) of the device status word; clears it."""
        need = C.c_int64(0)
        code = self.lib.piko_raster_status(self._h, C.byref(need))
        return code, need.value

    # -------------------------------------------------------------- passes
    def forward(self, scene: DeviceScene, fb: Optional[Framebuffer] = None, stream=None) -> Framebuffer:
        if fb is None:
            fb = Framebuffer.allocate(scene.width, scene.height, scene.shade_mode, scene.pos.device)
        cs, cf = scene.c_struct(), fb.c_struct()
        self._check(self.lib.piko_raster_forward(self._h, C.byref(cs), C.byref(cf), self._stream(stream)))
        return fb

    def forward_host(self, scene: HostScene, fb: Optional[Framebuffer] = None, stream=None) -> Framebuffer:
        """End-to-end frame through the C ABI with host buffers
        (piko_raster_forward_host): the library copies the scene's host
        arrays to the device, runs the forward pass and copies the key and
        colour (or G-buffer) into fb's host tensors, all on ``stream``.  fb
        defaults to pinned host tensors; the results are valid once the
        stream has passed the call."""
        if fb is None:
            fb = Framebuffer.allocate(scene.width, scene.height, scene.shade_mode, "cpu")
            for name in ("key", "rgba", "gbuf_normal", "gbuf_albedo"):
                if getattr(fb, name) is not None:
                    setattr(fb, name, getattr(fb, name).pin_memory())
        for name in ("key", "rgba", "gbuf_normal", "gbuf_albedo"):
            v = getattr(fb, name)
            if v is not None and (v.is_cuda or not v.is_contiguous()):
                raise ValueError(f"framebuffer {name} must be a contiguous CPU tensor")
        cs, cf = scene.c_struct(), fb.c_struct()
        self._check(self.lib.piko_raster_forward_host(self._h, C.byref(cs), C.byref(cf), self._stream(stream)))
        self._host_keepalive = (scene, fb)
        return fb

    def render_from_host(self, host_inputs: dict, scene: DeviceScene, fb: Framebuffer, key_out: torch.Tensor,
                         rgba_out: Optional[torch.Tensor] = None, stream=None) -> Framebuffer:
        """End-to-end frame from host memory: copies the named host tensors
        (pinned for asynchronous copies) into the scene's device tensors, runs
        the forward pass and copies the key (and rgba) back into host tensors,
        all on ``stream`` (default: the current stream), so that frames on two
        streams with two handles overlap their copies with each other's work."""
        s = torch.cuda.current_stream() if stream is None else stream
        with torch.cuda.stream(s):
            for name, t in host_inputs.items():
                getattr(scene, name).copy_(t, non_blocking=True)
            self.forward(scene, fb, s)
            key_out.copy_(fb.key, non_blocking=True)
            if rgba_out is not None and fb.rgba is not None:
                rgba_out.copy_(fb.rgba, non_blocking=True)
        return fb

    def deferred_light(self, fb: Framebuffer, lights: torch.Tensor, out: Optional[torch.Tensor] = None,
                       stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.height, self.width, 4), dtype=torch.float32, device=fb.key.device)
        lights = lights.contiguous()
        cf = fb.c_struct()
        self._check(self.lib.piko_raster_deferred_light(self._h, C.byref(cf), _ptr(lights), int(lights.shape[0]),
                                                        _ptr(out), self._stream(stream)))
        return out

    # -------------------------------------------------------------- batches
    def forward_batch(self, scenes, fbs=None, bin_sizes=None, schedules=None, stream=None):
        """All scenes in one pass (one persistent launch by default).
        bin_sizes: per-scene (w, h) pairs or None; schedules: per-scene names /
        PIKO_SCHED_* values or None.  Returns the list of framebuffers."""
        n = len(scenes)
        if fbs is None:
            fbs = [Framebuffer.allocate(s.width, s.height, s.shade_mode, s.pos.device) for s in scenes]
        cs = (L.PikoScene * n)(*[s.c_struct() for s in scenes])
        cf = (L.PikoFramebuffer * n)(*[f.c_struct() for f in fbs])
        bs = None
        if bin_sizes is not None:
            flat = [int(v) for wh in bin_sizes for v in wh]
            bs = (C.c_int32 * (2 * n))(*flat)
        sc = None
        if schedules is not None:
            sc = (C.c_int32 * n)(*[_SCHEDULES[x] if isinstance(x, str) else int(x) for x in schedules])
        self._check(self.lib.piko_raster_forward_batch(self._h, cs, n, cf, bs, sc, self._stream(stream)))
        self._batch_keepalive = (scenes, fbs)
        return fbs

    def backward_batch(self, scenes, fbs, dl_drgba, dcolor=None, dnormal=None, dlight=None, stream=None):
        """Gradients for the scenes of the last forward_batch (lists of tensors
        per scene; entries may be None)."""
        n = len(scenes)
        cs = (L.PikoScene * n)(*[s.c_struct() for s in scenes])
        cf = (L.PikoFramebuffer * n)(*[f.c_struct() for f in fbs])

        def ptrs(lst):
            if lst is None:
                return None
            return (C.c_void_p * n)(*[None if t is None else t.data_ptr() for t in lst])

        gl = [g.contiguous() for g in dl_drgba]
        self._check(self.lib.piko_raster_backward_batch(self._h, cs, n, cf, ptrs(gl), ptrs(dcolor), ptrs(dnormal),
                                                        ptrs(dlight), self._stream(stream)))
        return dcolor, dnormal, dlight

    def backward(self, scene: DeviceScene, fb: Framebuffer, dl_drgba: torch.Tensor, dcolor=None, dnormal=None,
                 dlight=None, stream=None):
        """Accumulates gradients into the given float32 tensors (any may be None)."""
        cs, cf = scene.c_struct(), fb.c_struct()
        g = dl_drgba.contiguous()
        self._check(self.lib.piko_raster_backward(self._h, C.byref(cs), C.byref(cf), _ptr(g), _ptr(dcolor),
                                                  _ptr(dnormal), _ptr(dlight), self._stream(stream)))
        return dcolor, dnormal, dlight
