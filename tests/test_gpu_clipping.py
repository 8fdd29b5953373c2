"""Near/far clipping (PIKO_OPT_CLIP) against the oracle's O16: keys bit for
bit, colours within 1e-5 and gradients within 1e-4 relative, for triangles
that cross the near and far planes or reach behind the eye."""
import dataclasses
import json
import os

import numpy as np
import pytest

import oracle
from paper_1404_6293_gb300 import scenes as S

pytestmark = pytest.mark.gpu

RGB_TOL = 1e-5
EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(autouse=True)
def _oracle_clipping():
    oracle.set_clipping(True)
    yield
    oracle.set_clipping(False)


def _torch():
    import torch
    return torch


def _render(scene, bins=16, schedule="dynamic", mvp=None, clip=1, persp=0, check=1):
    torch = _torch()
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene, Rasterizer
    r = Rasterizer(scene.width, scene.height, bins, bins, schedule)
    r.set_option(L.PIKO_OPT_CLIP, clip)
    r.set_option(L.PIKO_OPT_PERSPECTIVE, persp)
    r.set_option(L.PIKO_OPT_CHECK_CAPACITY, check)
    ds = DeviceScene.from_host(scene, mvp=mvp)
    fb = r.forward(ds)
    torch.cuda.synchronize()
    code, _ = r.status()
    return r, ds, fb, code


def _keys_equal(got, ref, what):
    bad = np.argwhere(got != ref)
    assert bad.size == 0, f"{what}: {len(bad)} keys differ, first at {tuple(bad[0][::-1])}"


def _crossing_scene(seed, T=400, W=160, H=112, mode=S.SHADE_GOURAUD):
    """Random triangles in clip space, some vertices beyond either plane or
    behind the eye (w < 0)."""
    rng = np.random.default_rng(seed)
    xy = rng.uniform(-1.3, 1.3, (3 * T, 2))
    w = rng.uniform(0.2, 2.0, 3 * T)
    w[rng.random(3 * T) < 0.1] *= -1.0
    z = rng.uniform(-1.6, 1.6, 3 * T) * np.abs(w)
    pos = np.stack([xy[:, 0] * w, xy[:, 1] * w, z, w], 1).astype(np.float32)
    col = rng.uniform(0, 1, (3 * T, 3)).astype(np.float32)
    nrm = rng.uniform(-1, 1, (3 * T, 3))
    nrm[:, 2] = -np.abs(nrm[:, 2]) - 0.3
    nrm = (nrm / np.linalg.norm(nrm, axis=1, keepdims=True)).astype(np.float32)
    return S.Scene(W, H, pos, np.arange(3 * T, dtype=np.int32).reshape(T, 3), color=col, normal=nrm,
                   light_dir=np.array([0.3, -0.4, -0.866], np.float32) if mode == S.SHADE_LAMBERT else None,
                   shade_mode=mode)


def test_near_plane_golden_8x8():
    with open(os.path.join(GOLDEN, "clip_near_8x8.json")) as f:
        g = json.load(f)
    s = S.Scene(8, 8, np.asarray(g["verts_clip"], np.float32), np.array([[0, 1, 2]], np.int32),
                color=np.asarray(g["colors"], np.float32))
    _, _, fb, code = _render(s, bins=8, clip=0)
    assert code == 0 and np.all(fb.key_numpy() == EMPTY)  # culled without clipping
    for sched in ("static", "dynamic", "hardware", "fused", "unfused"):
        _, _, fb, code = _render(s, bins=8, schedule=sched)
        assert code == 0
        key, rgba = fb.key_numpy(), fb.rgba.cpu().numpy()
        for y in range(8):
            for x in range(8):
                k = f"{x},{y}"
                if k in g["covered"]:
                    assert int(key[y, x]) == g["covered"][k] << 32, (sched, k)
                    assert np.abs(rgba[y, x, :3] - g["rgb"][k]).max() <= RGB_TOL, (sched, k)
                else:
                    assert key[y, x] == EMPTY, (sched, k)


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("bins,schedule", [(8, "static"), (16, "dynamic"), (16, "hardware"), (64, "dynamic"),
                                           (16, "fused"), (16, "unfused")])
def test_random_crossing_triangles_every_schedule(seed, bins, schedule):
    s = _crossing_scene(seed)
    assert oracle.clip_count(s) > 0
    ref, _ = oracle.raster_brute(s)
    _, _, fb, code = _render(s, bins, schedule)
    assert code == 0
    _keys_equal(fb.key_numpy(), ref, f"seed {seed} {bins} {schedule}")
    assert np.abs(fb.rgba.cpu().numpy() - oracle.shade(s, ref)).max() <= RGB_TOL


def _sphere_near_far(W=192, H=128, slices=60, stacks=40, dist=1.5, near=1.0, far=2.0):
    sph, _ = S.sphere_views(num_views=1, width=W, height=H, slices=slices, stacks=stacks)
    d = np.array([0.6, 0.3, 0.74])
    d /= np.linalg.norm(d)
    mvp = S._look_at_perspective(dist * d, [0.0, 0.0, 0.0], [0.0, 1.0, 0.0], 70.0, W / H, near, far)
    return dataclasses.replace(sph, mvp=mvp.astype(np.float32).ravel())


@pytest.mark.parametrize("persp", [0, 1])
def test_sphere_cut_by_both_planes(persp):
    """The camera's near plane cuts the front of the sphere and the far plane
    its back: the clipped rim is drawn instead of lost."""
    s = _sphere_near_far()
    assert oracle.clip_count(s) > 50
    ref, _ = oracle.raster_bbox(s, threads=4)
    with oracle.clipping(False):
        culled, _ = oracle.raster_bbox(s, threads=4)
    assert (ref != EMPTY).sum() > (culled != EMPTY).sum()
    for sched in ("hardware", "dynamic", "fused"):
        _, _, fb, code = _render(s, 16, sched, persp=persp)
        assert code == 0
        _keys_equal(fb.key_numpy(), ref, f"sphere {sched}")
        err = np.abs(fb.rgba.cpu().numpy() - oracle.shade(s, ref, perspective=bool(persp))).max()
        assert err <= RGB_TOL, (sched, err)


@pytest.mark.parametrize("shape", ["tile", "pixel"])
def test_clipped_gradients_match_oracle(shape):
    """Gradients through clipped winners (ray weights) in both backward forms:
    the tile form (few triangles per pixel) and the per-pixel form."""
    torch = _torch()
    if shape == "tile":
        s = _sphere_near_far(W=256, H=192, slices=40, stacks=24)
        assert 4 * s.num_triangles <= s.width * s.height
    else:
        s = _sphere_near_far(W=96, H=64, slices=80, stacks=50)
        assert 4 * s.num_triangles > s.width * s.height
    r, ds, fb, code = _render(s, 16, "dynamic")
    assert code == 0
    ref, _ = oracle.raster_bbox(s, threads=4)
    _keys_equal(fb.key_numpy(), ref, shape)
    tgt = S.target_image(s.width, s.height, seed=7)[0]
    g = np.zeros((s.height, s.width, 4))
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
        assert np.abs(got - want)[~big].max(initial=0) <= 1e-4 * scale


def test_no_crossing_is_unchanged_and_clip_off_still_culls():
    s = S.random_triangles(128, 96, 400, 14.0, seed=5)
    ref, _ = oracle.raster_brute(s)
    _, _, a, _ = _render(s, clip=1)
    _, _, b, _ = _render(s, clip=0)
    _keys_equal(a.key_numpy(), ref, "clip on")
    _keys_equal(b.key_numpy(), ref, "clip off")
    c = _crossing_scene(3)
    with oracle.clipping(False):
        ref_off, _ = oracle.raster_brute(c)
    _, _, fb, code = _render(c, clip=0)
    _keys_equal(fb.key_numpy(), ref_off, "crossing scene, clipping off")


def test_clip_list_grows_or_reports_overflow():
    """More sub-triangles than the first list holds (T / 8 + 1024): with the
    capacity check the list grows and the frame is exact, without it the
    frame reports PIKO_ERR_OVERFLOW and writes nothing."""
    torch = _torch()
    from paper_1404_6293_gb300 import _lib as L
    s = _crossing_scene(11, T=6000, W=128, H=96)
    n = oracle.clip_count(s)
    assert n > 6000 // 8 + 1024
    ref, _ = oracle.raster_bbox(s, threads=4)
    r, ds, fb, code = _render(s, 16, "dynamic", check=1)
    assert code == 0
    _keys_equal(fb.key_numpy(), ref, "after growth")
    r2, ds2, fb2, code2 = _render(s, 16, "dynamic", check=0)
    assert code2 == L.PIKO_ERR_OVERFLOW


def test_batch_rejects_clipping():
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene, PikoError, Rasterizer
    s = S.random_triangles(64, 64, 50, 8.0, seed=1)
    r = Rasterizer(64, 64)
    r.set_option(L.PIKO_OPT_CLIP, 1)
    with pytest.raises(PikoError):
        r.forward_batch([DeviceScene.from_host(s)])
