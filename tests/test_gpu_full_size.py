"""Parity at the full workload sizes, in the launch configurations bench.py
times, and under CUDA-graph replay.

Every frame is compared whole against the oracle: the 1080p heightfield
under every schedule the bench can time, all 64 sphere views (keys and
colour) plus one view's gradients, and all 256 scenes of the batch (keys and
colour).  The oracle's bounding-box form runs on all host cores; frames are
spread over a thread pool (the oracle's C calls release the interpreter
lock), so the whole file stays within a few minutes on the host.
"""
import concurrent.futures as cf
import dataclasses
import os

import numpy as np
import pytest

import oracle
from paper_1404_6293_gb300 import scenes as S

pytestmark = pytest.mark.gpu

RGB_TOL = 1e-5
CORES = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def _torch():
    import torch
    return torch


def _oracle_frames(scenes, mvps=None, with_rgba=True):
    """Oracle keys (and float64 colour) of many frames, in parallel."""
    mvps = mvps if mvps is not None else [None] * len(scenes)

    def one(i):
        key, st = oracle.raster_bbox(scenes[i], mvp=mvps[i], threads=1)
        assert st == 0
        return key, (oracle.shade(scenes[i], key, mvp=mvps[i]) if with_rgba else None)

    with cf.ThreadPoolExecutor(max_workers=CORES) as ex:
        return list(ex.map(one, range(len(scenes))))


def _check_frames(scenes, keys, rgbas, labels, mvps=None):
    """Compares every frame with the oracle (keys bit-exact, colour within
    1e-5), frames in parallel; raises on the first frame that differs."""
    mvps = mvps if mvps is not None else [None] * len(scenes)

    def one(i):
        key, st = oracle.raster_bbox(scenes[i], mvp=mvps[i], threads=1)
        assert st == 0
        _assert_keys(keys[i], key, labels[i])
        if rgbas is not None:
            err = np.abs(rgbas[i] - oracle.shade(scenes[i], key, mvp=mvps[i])).max()
            assert err <= RGB_TOL, (labels[i], err)
        return True

    with cf.ThreadPoolExecutor(max_workers=CORES) as ex:
        assert all(ex.map(one, range(len(scenes))))


def _assert_keys(got, ref, what):
    if not np.array_equal(got, ref):
        bad = np.argwhere(got != ref)
        y, x = bad[0]
        raise AssertionError(f"{what}: {len(bad)} keys differ, first at (x={x}, y={y}): "
                             f"gpu {int(got[y, x]):#x} oracle {int(ref[y, x]):#x}")


def _grad_check(g_gpu, g_ref, what):
    g_gpu = np.asarray(g_gpu, np.float64)
    scale = np.abs(g_ref).max()
    big = np.abs(g_ref) > 1e-3 * scale
    rel = np.abs(g_gpu - g_ref)[big] / np.abs(g_ref)[big]
    assert rel.max() <= 1e-4, (what, rel.max())
    assert np.abs(g_gpu - g_ref)[~big].max(initial=0) <= 1e-4 * scale, what


@pytest.mark.parametrize("bins,schedule", [(16, "hardware"), (16, "dynamic"), (16, "static"), (8, "hardware"),
                                           (32, "hardware"), (64, "dynamic")])
def test_heightfield_1080p_full_frame_bench_launches(bins, schedule):
    """The headline workload in the launch the bench times (16x16, one CTA
    per tile, the library's default threads), the other schedules and the
    bin sizes of the sweep: every key bit-exact, every colour within 1e-5."""
    torch = _torch()
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene, Framebuffer, Rasterizer
    s = S.heightfield()
    if not hasattr(test_heightfield_1080p_full_frame_bench_launches, "_ref"):
        key, _ = oracle.raster_bbox(s, threads=CORES)
        test_heightfield_1080p_full_frame_bench_launches._ref = (key, oracle.shade(s, key))
    ref, rgba_ref = test_heightfield_1080p_full_frame_bench_launches._ref
    r = Rasterizer(s.width, s.height, bins, bins, schedule)
    ds = DeviceScene.from_host(s)
    fb = Framebuffer.allocate(s.width, s.height, s.shade_mode)
    r.forward(ds, fb)
    assert r.status()[0] == 0
    r.set_option(L.PIKO_OPT_CHECK_CAPACITY, 0)  # the bench's timed form: no read-back
    fb.key.fill_(0)
    fb.rgba.fill_(-1.0)
    r.forward(ds, fb)
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    _assert_keys(fb.key_numpy(), ref, f"heightfield 1080p {bins}x{bins} {schedule}")
    assert np.abs(fb.rgba.cpu().numpy() - rgba_ref).max() <= RGB_TOL
    r.close()


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


def _sphere_batch(nv=64):
    torch = _torch()
    from paper_1404_6293_gb300.raster import DeviceScene, Framebuffer, Rasterizer
    sph, mvps = S.sphere_views(num_views=nv)
    W, H = sph.width, sph.height
    ds = DeviceScene.from_host(sph)
    mv = torch.from_numpy(mvps).cuda()
    views = [dataclasses.replace(ds, mvp=mv[v]) for v in range(nv)]
    key_all = torch.empty((nv, H, W), dtype=torch.int64, device="cuda")
    rgba_all = torch.empty((nv, H, W, 4), dtype=torch.float32, device="cuda")
    fbs = [Framebuffer(key_all[v], rgba_all[v]) for v in range(nv)]
    r = Rasterizer(W, H, 16, 16)
    return sph, mvps, ds, views, key_all, rgba_all, fbs, r


def test_sphere_64_views_full_size_every_view():
    """The 64 views at 512x512 as the bench renders them (one forward_batch,
    16x16 bins, dynamic): every view's keys bit-exact and colours within 1e-5."""
    torch = _torch()
    sph, mvps, ds, views, key_all, rgba_all, fbs, r = _sphere_batch()
    nv = len(views)
    r.forward_batch(views, fbs, [(16, 16)] * nv, ["dynamic"] * nv)
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    keys = key_all.cpu().numpy().view(np.uint64)
    rgba = rgba_all.cpu().numpy()
    _check_frames([sph] * nv, keys, rgba, [f"sphere view {v}" for v in range(nv)], list(mvps))


def test_sphere_512_view_gradients_full_size():
    """One 512x512 view of the 99.5k-triangle sphere: forward + L2-loss
    backward through the batch path the bench times (one view of the batch)
    and through the single-scene path, against the oracle's float64 colour,
    normal and light gradients (1e-4 relative)."""
    torch = _torch()
    from paper_1404_6293_gb300.raster import Rasterizer
    sph, mvps, ds, views, key_all, rgba_all, fbs, r = _sphere_batch(nv=4)
    W, H = sph.width, sph.height
    v = 2
    sv = S.Scene(W, H, sph.pos, sph.tris, color=sph.color, normal=sph.normal, mvp=mvps[v],
                 light_dir=sph.light_dir, shade_mode=sph.shade_mode)
    ref_key, _ = oracle.raster_bbox(sv, threads=CORES)
    rgba_ref = oracle.shade(sv, ref_key)
    tgt = S.target_image(W, H, seed=1240, views=4)[v]
    g = np.zeros((H, W, 4))
    g[..., :3] = 2.0 * (rgba_ref[..., :3] - tgt[..., :3])
    dc_ref, dn_ref, dl_ref = oracle.backward(sv, ref_key, g)
    gd = torch.from_numpy(g.astype(np.float32)).cuda()
    # batch path: the one view alone in a batch
    fb = r.forward_batch([views[v]], [fbs[v]], [(16, 16)], ["dynamic"])[0]
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    _assert_keys(fb.key_numpy(), ref_key, "sphere view gradients: batch forward")
    dc = torch.zeros_like(ds.color)
    dn = torch.zeros_like(ds.normal)
    dl = torch.zeros_like(ds.light_dir)
    r.backward_batch([views[v]], [fb], [gd], [dc], [dn], [dl])
    torch.cuda.synchronize()
    _grad_check(dc.cpu().numpy(), dc_ref, "batch dcolor")
    _grad_check(dn.cpu().numpy(), dn_ref, "batch dnormal")
    _grad_check(dl.cpu().numpy(), dl_ref, "batch dlight")
    # single-scene path
    rs = Rasterizer(W, H, 16, 16, "dynamic")
    fs = rs.forward(views[v])
    dc.zero_(); dn.zero_(); dl.zero_()
    rs.backward(views[v], fs, gd, dc, dn, dl)
    torch.cuda.synchronize()
    assert rs.status()[0] == 0
    _assert_keys(fs.key_numpy(), ref_key, "sphere view gradients: single forward")
    _grad_check(dc.cpu().numpy(), dc_ref, "single dcolor")
    _grad_check(dn.cpu().numpy(), dn_ref, "single dnormal")
    _grad_check(dl.cpu().numpy(), dl_ref, "single dlight")
    rs.close()


def test_batch_256_scenes_full_size_every_scene_and_launch_forms_agree():
    """All 256 scenes (10.4 M triangles, 120 M pixels) in one forward_batch at
    the setting the bench's tuner picks (32x32, dynamic): every scene's keys
    bit-exact and colours within 1e-5; the per-phase launch form agrees with
    the persistent one on every pixel."""
    torch = _torch()
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene, Rasterizer
    host = S.scene_batch(256)
    ds = [DeviceScene.from_host(s) for s in host]
    n = len(ds)
    bins, scheds = [(32, 32)] * n, ["dynamic"] * n
    r = Rasterizer(64, 64, 16, 16)
    fbs = r.forward_batch(ds, None, bins, scheds)
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    keys = [f.key_numpy() for f in fbs]
    rgbas = [f.rgba.cpu().numpy() for f in fbs]
    _check_frames(host, keys, rgbas, [f"batch scene {i} ({host[i].width}x{host[i].height}, "
                                      f"{host[i].num_triangles} triangles)" for i in range(n)])
    r.set_option(L.PIKO_OPT_BATCH_LAUNCH, 1)
    fbs2 = r.forward_batch(ds, None, bins, scheds)
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    for i in range(n):
        assert np.array_equal(keys[i], fbs2[i].key_numpy()), f"scene {i}: persistent and per-phase launches differ"


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
    refs = _oracle_frames(host, with_rgba=False)
    for i in range(n):
        assert torch.equal(direct[i], fbs[i].key), f"scene {i}: graph replay differs from the direct call"
        assert np.array_equal(fbs[i].key_numpy(), refs[i][0]), f"scene {i}: graph replay differs from the oracle"
