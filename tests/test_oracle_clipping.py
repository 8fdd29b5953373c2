"""Pins of the oracle's near/far clipping (O16), CPU only.

Clipping replaces the culls of O2/O3: a triangle crossing z = -w or z = w is
clipped in clip space, fanned, and its sub-triangles rasterize with the
original triangle's index; a clipped triangle shades from its original
vertices with the clip-space weights of each centre's ray.  Pinned against a
hand-derived 8x8 case, a band of a tilted full-screen quad that must be
covered exactly once, the unclipped definition where nothing crosses, the
bounding-box and scanline forms, and the ray/plane value of a linear
attribute on a floor that extends behind the camera.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1404_6293_gb300 import scenes as S

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(autouse=True)
def _clipping_off_afterwards():
    yield
    oracle.set_clipping(False)


def _scene(W, H, verts, tris, colors=None, mvp=None):
    return S.Scene(W, H, np.asarray(verts, np.float32), np.asarray(tris, np.int32).reshape(-1, 3),
                   color=None if colors is None else np.asarray(colors, np.float32),
                   mvp=None if mvp is None else np.asarray(mvp, np.float32).ravel())


def test_near_plane_golden_8x8():
    with open(os.path.join(GOLDEN, "clip_near_8x8.json")) as f:
        g = json.load(f)
    s = _scene(8, 8, g["verts_clip"], [[0, 1, 2]], g["colors"])
    key, st = oracle.raster_brute(s)
    assert st == 0 and np.all(key == EMPTY)          # clipping off: culled
    with oracle.clipping(True):
        assert oracle.clip_count(s) == 2
        key, st = oracle.raster_brute(s)
        assert st == 0
        rgba = oracle.shade(s, key)
    for y in range(8):
        for x in range(8):
            k = f"{x},{y}"
            if k in g["covered"]:
                assert int(key[y, x]) == (g["covered"][k] << 32), k
                assert np.allclose(rgba[y, x, :3], g["rgb"][k], rtol=0, atol=1e-12), (k, rgba[y, x])
                assert rgba[y, x, 3] == 1.0
            else:
                assert key[y, x] == EMPTY, k
                assert np.all(rgba[y, x] == 0.0)


def test_far_plane_mirror_of_the_golden():
    """z -> -z moves the clipped vertex behind the far plane instead: the
    same six pixels, with depths mirrored about the far plane (2^24 - 1 - Z)."""
    with open(os.path.join(GOLDEN, "clip_near_8x8.json")) as f:
        g = json.load(f)
    v = np.asarray(g["verts_clip"], np.float64)
    v[:, 2] = -v[:, 2]
    s = _scene(8, 8, v, [[0, 1, 2]], g["colors"])
    with oracle.clipping(True):
        key, _ = oracle.raster_brute(s)
    got = {f"{x},{y}": int(key[y, x] >> np.uint64(32)) for y in range(8) for x in range(8) if key[y, x] != EMPTY}
    # z = 0 -> 8388608 as before; z = +1 -> 16777215 at y = 4; Z linear in y:
    # 16777215 - 8388607 (y - 4) / 2, floored: 14680063 on row 4 (y = 4.5),
    # 10485759 on row 5 (y = 5.5)
    assert set(got) == set(g["covered"])
    for k in got:
        assert got[k] == (14680063 if k.endswith(",4") else 10485759), (k, got[k])


def test_tilted_quad_band_covered_exactly_once():
    """A full-screen quad on the plane z = 3y (w = 1) crosses both planes:
    clipped, it must cover the band |y_ndc| <= 1/3 once and nothing else."""
    W, H = 64, 48
    v = [[-1.5, -1.5, -4.5, 1], [1.5, -1.5, -4.5, 1], [1.5, 1.5, 4.5, 1], [-1.5, 1.5, 4.5, 1]]
    for diag in (0, 1):
        tris = [[0, 1, 2], [0, 2, 3]] if diag == 0 else [[0, 1, 3], [1, 2, 3]]
        s = _scene(W, H, v, tris)
        with oracle.clipping(True):
            key, cnt, st = oracle.raster_brute(s, with_count=True)
        assert st == 0
        yc = 1.0 - (np.arange(H) + 0.5) / H * 2.0
        inside = np.abs(yc) < 1.0 / 3.0 - 1e-3
        outside = np.abs(yc) > 1.0 / 3.0 + 1e-3
        assert np.all(cnt[inside, :] == 1), diag
        assert np.all(cnt[outside, :] == 0), diag
        assert np.all(cnt <= 1)


def test_no_crossing_means_no_change():
    s = S.random_triangles(96, 64, 300, 12.0, seed=41)
    ref, _ = oracle.raster_brute(s)
    rgba = oracle.shade(s, ref)
    with oracle.clipping(True):
        assert oracle.clip_count(s) == 0
        key, _ = oracle.raster_brute(s)
        assert np.array_equal(key, ref)
        assert np.array_equal(oracle.shade(s, key), rgba)


def _crossing_scene(seed, T=120, W=64, H=48):
    """Random triangles in clip space, some vertices beyond either plane or
    behind the eye (w < 0)."""
    rng = np.random.default_rng(seed)
    xy = rng.uniform(-1.3, 1.3, (3 * T, 2))
    w = rng.uniform(0.2, 2.0, 3 * T)
    w[rng.random(3 * T) < 0.1] *= -1.0
    z = rng.uniform(-1.6, 1.6, 3 * T) * np.abs(w)
    pos = np.stack([xy[:, 0] * w, xy[:, 1] * w, z, w], 1)
    col = rng.uniform(0, 1, (3 * T, 3))
    return _scene(W, H, pos, np.arange(3 * T).reshape(T, 3), col)


@pytest.mark.parametrize("seed", range(6))
def test_bbox_and_scanline_forms_agree_with_brute_force(seed):
    s = _crossing_scene(seed)
    with oracle.clipping(True):
        assert oracle.clip_count(s) > 0
        ref, _ = oracle.raster_brute(s)
        assert np.array_equal(oracle.raster_bbox(s, threads=3)[0], ref)
        assert np.array_equal(oracle.raster_scanline(s)[0], ref)
        pix = np.stack(np.meshgrid(np.arange(s.width), np.arange(s.height)), -1).reshape(-1, 2)[::7]
        k, _ = oracle.keys_at(s, pix)
        assert np.array_equal(k, ref[pix[:, 1], pix[:, 0]])


def test_clipped_floor_attribute_is_the_ray_plane_value():
    """A floor quad that reaches behind the camera (its far corners are in
    front, its near corners behind the eye): a colour channel equal to world
    x (affine in world space) must shade to the world x where each covered
    centre's ray meets the floor."""
    W, H = 64, 48
    eye = np.array([0.0, 1.0, 0.0])
    # look down the -z axis, slightly downwards
    f = np.array([0.0, -0.3, -1.0]); f /= np.linalg.norm(f)
    s_ = np.cross(f, [0, 1, 0]); s_ /= np.linalg.norm(s_)
    u = np.cross(s_, f)
    view = np.eye(4)
    view[0, :3], view[1, :3], view[2, :3] = s_, u, -f
    view[:3, 3] = -view[:3, :3] @ eye
    near, far, fov = 0.1, 50.0, 60.0
    t = 1.0 / np.tan(np.radians(fov) / 2)
    proj = np.zeros((4, 4))
    proj[0, 0], proj[1, 1] = t / (W / H), t
    proj[2, 2], proj[2, 3], proj[3, 2] = (far + near) / (near - far), 2 * far * near / (near - far), -1.0
    M = (proj @ view).astype(np.float32)
    corners = np.array([[-4, 0, 3, 1], [4, 0, 3, 1], [4, 0, -30, 1], [-4, 0, -30, 1]], np.float64)
    col = np.stack([corners[:, 0] / 8 + 0.5, np.zeros(4), np.zeros(4)], 1)
    s = _scene(W, H, corners, [[0, 1, 2], [0, 2, 3]], col, mvp=M)
    with oracle.clipping(True):
        key, _ = oracle.raster_brute(s)
        rgba = oracle.shade(s, key)
    covered = key != EMPTY
    assert covered.sum() > 0.3 * W * H
    Minv = np.linalg.inv(M.astype(np.float64))
    errs = []
    for py, px in zip(*np.nonzero(covered)):
        xn = (px + 0.5) / W * 2 - 1
        yn = 1 - (py + 0.5) / H * 2
        a = Minv @ np.array([xn, yn, -1.0, 1.0]); a = a[:3] / a[3]
        b = Minv @ np.array([xn, yn, 1.0, 1.0]); b = b[:3] / b[3]
        tt = a[1] / (a[1] - b[1])  # where the ray meets y = 0
        xw = a[0] + tt * (b[0] - a[0])
        errs.append(abs(rgba[py, px, 0] - (xw / 8 + 0.5)))
    assert max(errs) < 1e-4, max(errs)
