"""The other two mappings of the raster pipeline (Sec. 7.2's design space):
full fusion without tiling (PIKO_SCHED_FUSED) and the Baseline pipeline with
one kernel per stage (PIKO_SCHED_UNFUSED) give the oracle's keys bit for bit
and its colours within 1e-5, like the binned path."""
import numpy as np
import pytest

import oracle
from paper_1404_6293_gb300 import scenes as S

pytestmark = pytest.mark.gpu

RGB_TOL = 1e-5
MAPPINGS = ["fused", "unfused"]


def _torch():
    import torch
    return torch


def _run(scene, schedule, options=None, mvp=None):
    torch = _torch()
    from paper_1404_6293_gb300.raster import DeviceScene, Rasterizer
    r = Rasterizer(scene.width, scene.height, 16, 16, schedule)
    for k, v in (options or {}).items():
        r.set_option(k, v)
    ds = DeviceScene.from_host(scene, mvp=mvp)
    fb = r.forward(ds)
    torch.cuda.synchronize()
    code, _ = r.status()
    return r, ds, fb, code


def _keys_equal(got, ref, what):
    bad = np.argwhere(got != ref)
    assert bad.size == 0, f"{what}: {len(bad)} keys differ, first at {tuple(bad[0][::-1])}"


@pytest.mark.parametrize("mapping", MAPPINGS)
def test_random_triangles_gouraud(mapping):
    s = S.random_triangles()
    _, _, fb, code = _run(s, mapping)
    assert code == 0
    ref, _ = oracle.raster_brute(s)
    _keys_equal(fb.key_numpy(), ref, mapping)
    assert np.abs(fb.rgba.cpu().numpy() - oracle.shade(s, ref)).max() <= RGB_TOL


@pytest.mark.parametrize("mapping", MAPPINGS)
def test_heightfield_lambert_and_unclamped_colours(mapping):
    from paper_1404_6293_gb300 import _lib as L
    s = S.heightfield(320, 180, 80, 40, seed=5, with_color=True)
    ref, _ = oracle.raster_bbox(s, threads=4)
    for unclamped in (0, 1):
        _, _, fb, code = _run(s, mapping, {L.PIKO_OPT_UNCLAMPED: unclamped})
        assert code == 0
        _keys_equal(fb.key_numpy(), ref, f"{mapping} unclamped={unclamped}")
        err = np.abs(fb.rgba.cpu().numpy() - oracle.shade(s, ref, unclamped=bool(unclamped))).max()
        assert err <= RGB_TOL


@pytest.mark.parametrize("mapping", MAPPINGS)
def test_power_law_gbuffer_large_and_small_triangles(mapping):
    s = S.power_law_triangles(480, 270, 20_000, seed=9)
    _, _, fb, code = _run(s, mapping)
    assert code == 0
    ref, _ = oracle.raster_bbox(s, threads=4)
    _keys_equal(fb.key_numpy(), ref, mapping)
    gn, ga = oracle.shade(s, ref)
    for got, want in ((fb.gbuf_normal.cpu().numpy(), gn), (fb.gbuf_albedo.cpu().numpy(), ga)):
        g = got.astype(np.float64)
        r = want.view(np.float16).astype(np.float64)
        step = np.spacing(np.maximum(np.abs(g), np.abs(r)).astype(np.float16)).astype(np.float64)
        assert np.all(np.abs(g - r) <= step + 1e-6)


@pytest.mark.parametrize("mapping", MAPPINGS)
def test_sphere_view_perspective_correct(mapping):
    from paper_1404_6293_gb300 import _lib as L
    sph, mvps = S.sphere_views(num_views=2, width=256, height=192, slices=80, stacks=60)
    _, _, fb, code = _run(sph, mapping, {L.PIKO_OPT_PERSPECTIVE: 1}, mvp=mvps[1])
    assert code == 0
    ref, _ = oracle.raster_bbox(sph, mvp=mvps[1])
    _keys_equal(fb.key_numpy(), ref, mapping)
    err = np.abs(fb.rgba.cpu().numpy() - oracle.shade(sph, ref, mvp=mvps[1], perspective=True)).max()
    assert err <= RGB_TOL


@pytest.mark.parametrize("mapping", MAPPINGS)
def test_empty_bad_index_and_degenerate(mapping):
    from paper_1404_6293_gb300 import _lib as L
    s = S.random_triangles(64, 48, 40, 10.0, seed=21)
    s.tris = s.tris.copy()
    s.tris[3] = [0, 1, 10_000]  # outside [0, V): culled and reported
    s.tris[5] = [7, 7, 7]       # zero area
    _, _, fb, code = _run(s, mapping)
    assert code == L.PIKO_ERR_BAD_INDEX
    ref, st = oracle.raster_brute(s)
    assert st == oracle.BAD_INDEX
    _keys_equal(fb.key_numpy(), ref, mapping)
    empty = S.Scene(64, 48, np.zeros((0, 4), np.float32), np.zeros((0, 3), np.int32),
                    color=np.zeros((0, 3), np.float32))
    _, _, fb, code = _run(empty, mapping)
    assert code == 0
    assert np.all(fb.key_numpy() == np.uint64(0xFFFFFFFFFFFFFFFF))
    assert np.all(fb.rgba.cpu().numpy() == 0)


def test_unfused_fragment_buffer_grows_or_reports_overflow():
    """Depth complexity far above two per pixel: with the capacity check the
    fragment buffer grows and the frame is exact; without it the frame
    reports PIKO_ERR_OVERFLOW."""
    torch = _torch()
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene, Rasterizer
    s = S.random_triangles(64, 64, 400, 90.0, seed=23)  # each triangle covers much of the screen
    ref, _ = oracle.raster_brute(s)
    r = Rasterizer(64, 64, 16, 16, "unfused")
    ds = DeviceScene.from_host(s)
    fb = r.forward(ds)
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    _keys_equal(fb.key_numpy(), ref, "unfused after growth")
    assert np.abs(fb.rgba.cpu().numpy() - oracle.shade(s, ref)).max() <= RGB_TOL
    r2 = Rasterizer(64, 64, 16, 16, "unfused")
    r2.set_option(L.PIKO_OPT_CHECK_CAPACITY, 0)
    fb2 = r2.forward(ds)
    torch.cuda.synchronize()
    assert r2.status()[0] == L.PIKO_ERR_OVERFLOW
    # the next frame after the first one sized the buffer through r is exact on r
    r.set_option(L.PIKO_OPT_CHECK_CAPACITY, 0)
    fb3 = r.forward(ds)
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    _keys_equal(fb3.key_numpy(), ref, "unfused, capacity check off, sized")


@pytest.mark.parametrize("mapping", MAPPINGS)
def test_backward_after_other_mapping_matches_oracle(mapping):
    """The keys are the binned path's, so the backward pass works unchanged."""
    torch = _torch()
    s = S.random_triangles(128, 96, 300, 14.0, seed=31, shade_mode=S.SHADE_LAMBERT, with_normals=True)
    s.light_dir = np.array([0.3, -0.4, -0.866], np.float32)
    r, ds, fb, code = _run(s, mapping)
    assert code == 0
    ref, _ = oracle.raster_brute(s)
    _keys_equal(fb.key_numpy(), ref, mapping)
    tgt = S.target_image(128, 96, seed=2)[0]
    g = np.zeros((96, 128, 4))
    g[..., :3] = 2.0 * (oracle.shade(s, ref)[..., :3] - tgt[..., :3])
    dc, dn, dl = oracle.backward(s, ref, g)
    V = s.num_vertices
    dcg = torch.zeros((V, 3), device="cuda")
    dng = torch.zeros((V, 3), device="cuda")
    dlg = torch.zeros(3, device="cuda")
    r.backward(ds, fb, torch.from_numpy(g.astype(np.float32)).cuda(), dcg, dng, dlg)
    torch.cuda.synchronize()
    for got, want in ((dcg, dc), (dng, dn), (dlg, dl)):
        got = got.cpu().numpy().astype(np.float64)
        scale = np.abs(want).max()
        big = np.abs(want) > 1e-3 * scale
        assert (np.abs(got - want)[big] / np.abs(want)[big]).max() <= 1e-4
