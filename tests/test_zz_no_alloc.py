"""The allocation-free forward entry point against the oracle and the ordinary
forward pass.

piko_raster_forward_noalloc serves callers that may not allocate GPU memory:
work recorded into a stream capture that must not add allocations, plugins
whose host application owns the device allocator, and real-time loops that
cannot pay for cudaMalloc's implicit synchronisation.  Its scratch is one
fixed array inside the library that every call shares, so these tests also
run calls of different sizes back to back (the array keeps what the last
call left), push the bin lists past the array's capacity, and check that
free device memory does not move.

This file is collected last so that a run stopping at the first failure has
run every other test already; it also passes on its own in a fresh process.
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


def _oracle(scene):
    import oracle
    key, st = oracle.raster_bbox(scene, threads=8)
    assert st == 0
    return key, oracle.shade(scene, key)


def _run_and_check(lib, scene, ds, bw, bh, sched, ref_key, ref_rgba, label):
    import torch
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import Framebuffer
    fb = Framebuffer.allocate(scene.width, scene.height, scene.shade_mode)
    fb.key.fill_(0)
    fb.rgba.fill_(-1.0)
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    assert _noalloc(lib, ds, fb, bw, bh, sched, status) == L.PIKO_OK, label
    torch.cuda.synchronize()
    assert int(status.item()) == L.PIKO_OK, label
    assert np.array_equal(fb.key_numpy(), ref_key), f"{label}: keys differ from the oracle"
    assert np.abs(fb.rgba.cpu().numpy() - ref_rgba).max() <= RGB_TOL, label


def test_noalloc_forward_matches_forward_and_oracle_on_two_calls_in_a_row():
    import torch
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene, Framebuffer, Rasterizer
    lib = L.load()
    cases = [
        (S.random_triangles(256, 256, 1000, 40.0, seed=1235), 16, 16, L.PIKO_SCHED_STATIC),
        (S.heightfield(320, 180, 80, 40, seed=5), 8, 8, L.PIKO_SCHED_DYNAMIC),  # Lambert
        (S.heightfield(320, 180, 80, 40, seed=6, with_color=True), 32, 16, L.PIKO_SCHED_HARDWARE),
    ]
    for scene, bw, bh, sched in cases:
        ds = DeviceScene.from_host(scene)
        ref = Rasterizer(scene.width, scene.height, bw, bh, sched).forward(ds)
        torch.cuda.synchronize()
        ref_key, ref_rgba = ref.key_numpy(), ref.rgba.cpu().numpy()
        okey, orgba = _oracle(scene)
        assert np.array_equal(ref_key, okey)
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        for call in range(2):  # the second call reuses the scratch the first one left behind
            fb = Framebuffer.allocate(scene.width, scene.height, scene.shade_mode)
            fb.key.fill_(0)
            fb.rgba.fill_(-1.0)
            status.fill_(-1)
            assert _noalloc(lib, ds, fb, bw, bh, sched, status) == L.PIKO_OK
            torch.cuda.synchronize()
            assert int(status.item()) == L.PIKO_OK
            got_key, got_rgba = fb.key_numpy(), fb.rgba.cpu().numpy()
            assert np.array_equal(got_key, ref_key), f"call {call}"
            assert np.abs(got_rgba - ref_rgba).max() <= RGB_TOL
            assert np.abs(got_rgba - orgba).max() <= RGB_TOL


def test_noalloc_many_tiles_after_few_tiles_and_back():
    """16,384 tiles (eight scan chunks of 2,048 tiles), then 928 tiles (one
    chunk), then 16,384 again: the scan states a large call leaves in the
    shared array are cleared, not read, by the calls after it."""
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene
    lib = L.load()
    big = S.random_triangles(1024, 1024, 20000, 6.0, seed=71)
    small = S.random_triangles(256, 230, 800, 10.0, seed=72)
    refs = {id(sc): _oracle(sc) for sc in (big, small)}
    dss = {id(sc): DeviceScene.from_host(sc) for sc in (big, small)}
    seq = [(big, 8, 8, L.PIKO_SCHED_DYNAMIC), (small, 8, 8, L.PIKO_SCHED_STATIC),
           (big, 8, 8, L.PIKO_SCHED_HARDWARE), (small, 16, 16, L.PIKO_SCHED_DYNAMIC),
           (big, 8, 8, L.PIKO_SCHED_STATIC)]
    for n, (sc, bw, bh, sched) in enumerate(seq):
        k, rgba = refs[id(sc)]
        _run_and_check(lib, sc, dss[id(sc)], bw, bh, sched, k, rgba, f"call {n} ({sc.width}x{sc.height})")


def test_noalloc_overflow_is_reported_and_leaves_the_framebuffer_untouched():
    """More (triangle, tile) pairs than the array's bin lists hold: the call
    reports PIKO_ERR_OVERFLOW through status_out and Process writes nothing;
    the next call that fits is exact again."""
    import torch
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene, Framebuffer
    lib = L.load()
    dense = S.random_triangles(1024, 1024, 20000, 96.0, seed=73)  # about 2.4 M (triangle, 8x8 tile) pairs
    ds = DeviceScene.from_host(dense)
    fb = Framebuffer.allocate(1024, 1024)
    fb.key.fill_(12345)
    fb.rgba.fill_(7.0)
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    assert _noalloc(lib, ds, fb, 8, 8, L.PIKO_SCHED_STATIC, status) == L.PIKO_OK
    torch.cuda.synchronize()
    assert int(status.item()) == L.PIKO_ERR_OVERFLOW
    assert bool((fb.key == 12345).all()) and bool((fb.rgba == 7.0).all())
    ok = S.random_triangles(256, 256, 1000, 40.0, seed=1235)
    k, rgba = _oracle(ok)
    _run_and_check(lib, ok, DeviceScene.from_host(ok), 16, 16, L.PIKO_SCHED_STATIC, k, rgba, "after overflow")


def test_noalloc_leaves_free_device_memory_unchanged():
    """After the first call (which looks up the array's address), further
    calls of any size allocate no device memory."""
    import torch
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene, Framebuffer
    lib = L.load()
    scenes = [S.random_triangles(1024, 1024, 20000, 6.0, seed=74), S.heightfield(320, 180, 80, 40, seed=5)]
    dss = [DeviceScene.from_host(s) for s in scenes]
    fbs = [Framebuffer.allocate(s.width, s.height, s.shade_mode) for s in scenes]
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert _noalloc(lib, dss[0], fbs[0], 8, 8, 0, status) == L.PIKO_OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        for ds, fb in zip(dss, fbs):
            assert _noalloc(lib, ds, fb, 8, 8, 1, status) == L.PIKO_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert int(status.item()) == L.PIKO_OK


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
