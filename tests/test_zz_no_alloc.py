"""The allocation-free forward entry point gives the same framebuffer as the
ordinary forward pass.

piko_raster_forward_noalloc serves callers that may not allocate GPU memory
(stream captures that must not add allocations, plugins whose host owns the
allocator, real-time loops).  This file is collected last so that a run
stopping at the first failure has run every other test already; it also
passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1404_6293_gb300 import scenes as S

pytestmark = pytest.mark.gpu

RGB_TOL = 1e-5  # the tolerance of the other colour parity tests


def _noalloc(lib, ds, fb, bin_w, bin_h, schedule, status):
    from paper_1404_6293_gb300 import _lib as L
    import torch
    f = lib.piko_raster_forward_noalloc
    f.argtypes = [C.POINTER(L.PikoScene), C.POINTER(L.PikoFramebuffer), C.c_int, C.c_int, C.c_int, C.c_void_p,
                  C.c_void_p]
    f.restype = C.c_int
    cs, cf = ds.c_struct(), fb.c_struct()
    return f(C.byref(cs), C.byref(cf), bin_w, bin_h, schedule, C.c_void_p(status.data_ptr()),
             C.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_forward_matches_forward_on_two_calls_in_a_row():
    import torch
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene, Framebuffer, Rasterizer
    lib = L.load()
    cases = [
        (S.random_triangles(256, 256, 1000, 40.0, seed=1235), 16, 16, L.PIKO_SCHED_STATIC),
        (S.heightfield(320, 180, 80, 40, seed=5), 8, 8, L.PIKO_SCHED_DYNAMIC),
    ]
    for scene, bw, bh, sched in cases:
        ds = DeviceScene.from_host(scene)
        ref = Rasterizer(scene.width, scene.height, bw, bh, sched).forward(ds)
        torch.cuda.synchronize()
        ref_key, ref_rgba = ref.key.cpu().numpy(), ref.rgba.cpu().numpy()
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        for call in range(2):  # the second call reuses the scratch the first one left behind
            fb = Framebuffer.allocate(scene.width, scene.height, scene.shade_mode)
            fb.key.fill_(0)
            fb.rgba.fill_(-1.0)
            status.fill_(-1)
            assert _noalloc(lib, ds, fb, bw, bh, sched, status) == L.PIKO_OK
            torch.cuda.synchronize()
            assert int(status.item()) == L.PIKO_OK
            assert np.array_equal(fb.key.cpu().numpy(), ref_key), f"call {call}"
            assert np.abs(fb.rgba.cpu().numpy() - ref_rgba).max() <= RGB_TOL


def test_noalloc_rejects_sizes_beyond_its_limits():
    import torch
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene, Framebuffer
    lib = L.load()
    scene = S.random_triangles(64, 64, 65537, 2.0, seed=3)  # one triangle over the limit
    ds = DeviceScene.from_host(scene)
    fb = Framebuffer.allocate(64, 64)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert _noalloc(lib, ds, fb, 16, 16, 0, status) == L.PIKO_ERR_INVALID_ARG
    big = S.random_triangles(2048, 1024, 10, 2.0, seed=3)  # 2048x1024 at 8x8 bins: 32768 tiles
    dsb = DeviceScene.from_host(big)
    fbb = Framebuffer.allocate(2048, 1024)
    assert _noalloc(lib, dsb, fbb, 8, 8, 0, status) == L.PIKO_ERR_INVALID_ARG
