"""piko_raster_forward_host: a scene in host memory in, a framebuffer in host
memory out, through the C ABI.  Keys bit-exact against the oracle and equal
to the device-memory forward; colours within 1e-5 of the oracle and of the
device-memory forward, G-buffer words within one binary16 step of it.  (Two
calls of one handle may shade a pixel once from its tile's shared record
and once from global memory -- the record area is sized from the previous
frame -- which rounds in a different order.)"""
import numpy as np
import pytest

import oracle
from paper_1404_6293_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def _run(scene, pin=True, sched="dynamic"):
    import torch
    from paper_1404_6293_gb300.raster import DeviceScene, Framebuffer, HostScene, Rasterizer
    r = Rasterizer(scene.width, scene.height, 16, 16, sched)
    hs = HostScene.from_host(scene, pin=pin)
    side = torch.cuda.Stream()
    fb_h = r.forward_host(hs, stream=side)
    side.synchronize()
    assert r.status()[0] == 0
    fb_d = r.forward(DeviceScene.from_host(scene))
    torch.cuda.synchronize()
    return r, fb_h, fb_d


@pytest.mark.parametrize("pin", [True, False])
def test_forward_host_lambert_with_matrix(pin):
    s = S.heightfield(160, 120, 60, 40, seed=91, with_color=True)
    r, fh, fd = _run(s, pin=pin)
    ref, _ = oracle.raster_brute(s)
    assert np.array_equal(fh.key.numpy().view(np.uint64), ref)
    assert np.array_equal(fh.key.numpy(), fd.key.cpu().numpy())
    assert np.abs(fh.rgba.numpy() - fd.rgba.cpu().numpy()).max() <= 1e-5
    assert np.abs(fh.rgba.numpy() - oracle.shade(s, ref)).max() <= 1e-5
    r.close()


def test_forward_host_gbuffer_and_growth():
    import torch
    from paper_1404_6293_gb300.raster import DeviceScene, HostScene, Rasterizer
    small = S.power_law_triangles(192, 128, 300, seed=92)
    big = S.power_law_triangles(192, 128, 3000, seed=93)
    r = Rasterizer(192, 128, 16, 16, "hardware")
    rd = Rasterizer(192, 128, 16, 16, "hardware")
    for s in (small, big, small):  # the device buffers grow on the second call
        fb = r.forward_host(HostScene.from_host(s))
        fd = rd.forward(DeviceScene.from_host(s))
        torch.cuda.synchronize()
        assert r.status()[0] == 0 and rd.status()[0] == 0
        ref, _ = oracle.raster_brute(s)
        assert np.array_equal(fb.key.numpy().view(np.uint64), ref)
        for a, b in ((fb.gbuf_normal, fd.gbuf_normal), (fb.gbuf_albedo, fd.gbuf_albedo)):
            a = a.float().numpy()
            b = b.cpu().float().numpy()
            step = np.maximum(np.abs(b), 2.0 ** -14) * 2.0 ** -10  # one binary16 step (normal range)
            assert (np.abs(a - b) <= step + 1e-7).all()
    r.close()
    rd.close()


def test_forward_host_rejects_size_mismatch():
    from paper_1404_6293_gb300.raster import HostScene, PikoError, Rasterizer
    s = S.random_triangles(64, 48, 20, 6.0, seed=94)
    r = Rasterizer(64, 64)
    with pytest.raises(PikoError):
        r.forward_host(HostScene.from_host(s))
    r.close()


def test_forward_host_rejects_missing_attributes_and_renders_empty_scene():
    import torch
    from paper_1404_6293_gb300.raster import HostScene, PikoError, Rasterizer
    s = S.random_triangles(64, 48, 20, 6.0, seed=95)
    r = Rasterizer(64, 48)
    hs = HostScene.from_host(s)
    hs.color = None  # Gouraud without colours
    with pytest.raises(PikoError):
        r.forward_host(hs)
    empty = HostScene.from_host(s)
    empty.tris = empty.tris[:0].contiguous()
    fb = r.forward_host(empty)
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    assert (fb.key.numpy().view(np.uint64) == np.uint64(0xFFFFFFFFFFFFFFFF)).all()
    assert (fb.rgba.numpy() == 0).all()
    r.close()
