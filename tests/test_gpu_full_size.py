"""Parity at the full workload sizes, in the launch configurations bench.py
times, and under CUDA-graph replay.

Full frames the oracle can afford are compared whole (tests/test_gpu_parity.py
does the 1080p heightfield and power-law frames); here the 64 sphere views
and the 256-scene batch are checked on seeded samples of pixels that the
oracle evaluates one by one (brute force over every triangle), plus
properties that hold at any size (the persistent and the per-phase batch
launches agree on every pixel; a graph replay equals a direct call).
"""
import numpy as np
import pytest

import oracle
from paper_1404_6293_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _sample_pixels(W, H, n, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, W, n), rng.integers(0, H, n)], axis=1).astype(np.int32)


def _check_samples(key_gpu, scene, n, seed, what, mvp=None):
    pix = _sample_pixels(scene.width, scene.height, n, seed)
    ref, _ = oracle.keys_at(scene, pix, mvp=mvp)
    got = key_gpu[pix[:, 1], pix[:, 0]]
    bad = np.nonzero(got != ref)[0]
    assert bad.size == 0, (f"{what}: {bad.size} of {n} sampled keys differ, first at {tuple(pix[bad[0]])}: "
                           f"gpu {int(got[bad[0]]):#x} oracle {int(ref[bad[0]]):#x}")


def test_forward_graph_replay_with_new_camera_matches_oracle():
    torch = _torch()
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene, Framebuffer, Rasterizer
    sph, mvps = S.sphere_views(num_views=3, width=256, height=192, slices=80, stacks=60)
    r = Rasterizer(sph.width, sph.height, 16, 16, "static")
    ds = DeviceScene.from_host(sph, mvp=mvps[0])
    fb = Framebuffer.allocate(sph.width, sph.height, sph.shade_mode)
    r.forward(ds, fb)
    code, need = r.status()
    assert code == 0
    r.reserve(sph.num_vertices, sph.num_triangles, 4 * need + 4096)
    r.set_option(L.PIKO_OPT_CHECK_CAPACITY, 0)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        r.forward(ds, fb, side)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        r.forward(ds, fb)
    torch.cuda.synchronize()
    for v in (1, 2, 0):
        ds.mvp.copy_(torch.from_numpy(np.ascontiguousarray(mvps[v], np.float32).reshape(16)))
        g.replay()
        torch.cuda.synchronize()
        assert r.status()[0] == 0
        ref, _ = oracle.raster_bbox(sph, mvp=mvps[v])
        got = fb.key_numpy()
        assert np.array_equal(got, ref), f"view {v}: {int((got != ref).sum())} keys differ after replay"


def test_sphere_64_views_full_size_sampled():
    torch = _torch()
    from paper_1404_6293_gb300.raster import DeviceScene, Framebuffer, Rasterizer
    sph, mvps = S.sphere_views(num_views=64)
    r = Rasterizer(sph.width, sph.height, 16, 16, "static")
    ds = DeviceScene.from_host(sph)
    mv = torch.from_numpy(mvps).cuda()
    fbs = [Framebuffer.allocate(sph.width, sph.height, sph.shade_mode) for _ in range(64)]
    for v in range(64):
        ds.mvp = mv[v]
        r.forward(ds, fbs[v])
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    for v in range(0, 64, 9):
        _check_samples(fbs[v].key_numpy(), sph, 96, 100 + v, f"sphere view {v}", mvp=mvps[v])


def test_batch_256_scenes_full_size_sampled_and_launch_forms_agree():
    torch = _torch()
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene, Rasterizer
    host = S.scene_batch(256)
    ds = [DeviceScene.from_host(s) for s in host]
    n = len(ds)
    bins, scheds = [(32, 32)] * n, ["dynamic"] * n  # the bench's tuned setting
    r = Rasterizer(64, 64, 16, 16)
    fbs = r.forward_batch(ds, None, bins, scheds)
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    keys = [f.key.clone() for f in fbs]
    for i in range(0, n, 16):
        _check_samples(fbs[i].key_numpy(), host[i], 48, 200 + i, f"batch scene {i}")
    r.set_option(L.PIKO_OPT_BATCH_LAUNCH, 1)
    fbs2 = r.forward_batch(ds, None, bins, scheds)
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    for i in range(n):
        assert torch.equal(keys[i], fbs2[i].key), f"scene {i}: persistent and per-phase launches differ"


def test_batch_graph_replay_equals_direct_call():
    torch = _torch()
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene, Rasterizer
    host = S.scene_batch(24, tmax=20_000, side_max=512, seed=77)
    ds = [DeviceScene.from_host(s) for s in host]
    n = len(ds)
    bins = [(16, 16), (32, 32)] * (n // 2)
    scheds = ["static", "dynamic", "dynamic", "static"] * (n // 4)
    r = Rasterizer(64, 64, 16, 16)
    fbs = r.forward_batch(ds, None, bins, scheds)
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    direct = [f.key.clone() for f in fbs]
    for f in fbs:
        f.key.fill_(0)
    r.set_option(L.PIKO_OPT_CHECK_CAPACITY, 0)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        r.forward_batch(ds, fbs, bins, scheds, stream=side)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        r.forward_batch(ds, fbs, bins, scheds)
    for f in fbs:
        f.key.fill_(0)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    for i in range(n):
        assert torch.equal(direct[i], fbs[i].key), f"scene {i}: graph replay differs from the direct call"
        ref, _ = oracle.raster_bbox(host[i])
        assert np.array_equal(fbs[i].key_numpy(), ref), f"scene {i}: graph replay differs from the oracle"
