"""Pins of the oracle's perspective-correct reading (O15), on the CPU.

b'_i = (b_i / w_i) / sum_j (b_j / w_j) with w_i the clip w of each vertex.
- With equal w, O15 reduces to the screen-space barycentrics of O11.
- An attribute that is affine in world space equals, at each covered pixel,
  the same affine function evaluated where the pixel centre's ray meets the
  triangle's plane. That hit point is computed here by unprojecting through
  the inverse camera matrix, which is independent of O15's formula. The
  screen-space form misses it by far more.
- Gradients with O15 match float64 central differences of the loss.
- A hand-derived case gives b' = (4/7, 2/7, 1/7) at a triangle's screen
  centroid with w = (1, 2, 4).
"""
import numpy as np

import oracle
from paper_1404_6293_gb300 import scenes as S

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


def _ids(key):
    out = (key & np.uint64(0xFFFFFFFF)).astype(np.int64)
    out[key == EMPTY] = -1
    return out


def test_equal_w_reduces_to_screen_space():
    s = S.random_triangles(64, 64, 60, 14.0, seed=31)
    key, _ = oracle.raster_brute(s)
    a = oracle.shade(s, key)
    b = oracle.shade(s, key, perspective=True)
    assert (key != EMPTY).sum() > 500
    assert np.abs(a - b).max() < 1e-12
    # scaling a vertex's homogeneous coordinates by c > 0 moves nothing on
    # screen but divides its weight by c: with every vertex scaled alike the
    # image is unchanged
    s2 = S.Scene(s.width, s.height, (s.pos.astype(np.float64) * 4.0).astype(np.float32), s.tris, color=s.color)
    key2, _ = oracle.raster_brute(s2)
    assert np.array_equal(key2, key)
    assert np.abs(oracle.shade(s2, key2, perspective=True) - a).max() < 1e-12


def _floor_scene(W=96, H=96):
    """Two large triangles of a receding floor (y = 0 in world space) seen by a
    tilted perspective camera, with colours affine in the world position."""
    world = np.array([[-1.5, 0.0, -0.5], [1.5, 0.0, -0.5], [1.5, 0.0, -6.0], [-1.5, 0.0, -6.0]])
    tris = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    M = S._look_at_perspective([0.0, 1.0, 1.0], [0.0, 0.0, -3.0], [0.0, 1.0, 0.0], 60.0, W / H, 0.1, 20.0)
    Ac = np.array([[0.25, 0.0, 0.05], [0.0, 0.0, -0.15], [0.1, 0.0, 0.1]])
    bc = np.array([0.5, 0.1, 0.8])
    color = world @ Ac.T + bc
    pos = np.concatenate([world, np.ones((4, 1))], 1).astype(np.float32)
    s = S.Scene(W, H, pos, tris, color=color.astype(np.float32), mvp=M.astype(np.float32).reshape(16))
    return s, M, world, Ac, bc


def _ray_hit_colour(M, world, tri, px, py, W, H, Ac, bc):
    Minv = np.linalg.inv(M.astype(np.float32).astype(np.float64))
    xn = (px + 0.5) / W * 2.0 - 1.0
    yn = 1.0 - (py + 0.5) / H * 2.0
    a = Minv @ np.array([xn, yn, -1.0, 1.0])
    b = Minv @ np.array([xn, yn, 1.0, 1.0])
    p0, p1 = a[:3] / a[3], b[:3] / b[3]
    v0, v1, v2 = world[tri[0]], world[tri[1]], world[tri[2]]
    nrm = np.cross(v1 - v0, v2 - v0)
    t = np.dot(v0 - p0, nrm) / np.dot(p1 - p0, nrm)
    hit = p0 + t * (p1 - p0)
    return Ac @ hit + bc


def test_world_affine_attribute_is_the_ray_hit_value():
    s, M, world, Ac, bc = _floor_scene()
    key, _ = oracle.raster_brute(s)
    ids = _ids(key)
    persp = oracle.shade(s, key, perspective=True)
    affine = oracle.shade(s, key)
    ys, xs = np.nonzero(ids >= 0)
    assert ys.size > 2000
    err_p = err_a = 0.0
    for py, px in zip(ys[::7], xs[::7]):
        want = _ray_hit_colour(M, world, s.tris[ids[py, px]], px, py, s.width, s.height, Ac, bc)
        err_p = max(err_p, np.abs(persp[py, px, :3] - want).max())
        err_a = max(err_a, np.abs(affine[py, px, :3] - want).max())
    # snapped vertices (1/256 px) and float32 transforms bound the residual
    assert err_p < 2e-3, err_p
    # screen-space interpolation of the same attribute is visibly wrong
    assert err_a > 20 * err_p and err_a > 0.02, (err_a, err_p)


def test_perspective_gradients_match_central_differences():
    sph, mvps = S.sphere_views(num_views=1, width=48, height=48, slices=14, stacks=10, seed=9)
    M = mvps[0]
    key, _ = oracle.raster_brute(sph, mvp=M)
    tgt = S.target_image(48, 48, seed=4)[0]
    rgba = oracle.shade(sph, key, mvp=M, perspective=True)
    g = np.zeros((48, 48, 4))
    g[..., :3] = 2.0 * (rgba[..., :3] - tgt[..., :3])
    dc, dn, dl = oracle.backward(sph, key, g, mvp=M, perspective=True)
    col = sph.color.astype(np.float64)
    nrm = sph.normal.astype(np.float64)
    L = sph.light_dir.astype(np.float64)

    def fd(which, idx):
        c, n, l = col.copy(), nrm.copy(), L.copy()
        arr = {"c": c, "n": n, "l": l}[which]
        th = arr.flat[idx]
        h = 1e-6 * max(1.0, abs(th))
        arr.flat[idx] = th + h
        lp = oracle.loss(sph, key, tgt, mvp=M, color=c, normal=n, light=l, perspective=True)
        arr.flat[idx] = th - h
        lm = oracle.loss(sph, key, tgt, mvp=M, color=c, normal=n, light=l, perspective=True)
        return (lp - lm) / (2 * h)

    rng = np.random.default_rng(5)
    used = np.unique(sph.tris[np.unique(_ids(key)[key != EMPTY])])
    params = np.array([3 * v + ch for v in used for ch in range(3)])
    assert params.size >= 48
    for which, an in (("c", dc), ("n", dn)):
        scale = np.abs(an).max()
        assert scale > 0
        for idx in rng.choice(params, 48, replace=False):
            v, ch = divmod(int(idx), 3)
            assert abs(fd(which, int(idx)) - an[v, ch]) <= 1e-4 * max(abs(an[v, ch]), 1e-3 * scale) + 1e-9
    for ch in range(3):
        assert abs(fd("l", ch) - dl[ch]) <= 1e-4 * max(abs(dl[ch]), 1e-3 * np.abs(dl).max())
    # and the perspective gradients differ from the screen-space ones
    dc_a, _, _ = oracle.backward(sph, key, g, mvp=M)
    assert np.abs(dc_a - dc).max() > 1e-3 * np.abs(dc).max()


def test_centroid_with_w_1_2_4_is_4_2_1_sevenths():
    """Hand-derived: at a pixel centre that is the triangle's screen
    centroid, b = (1/3, 1/3, 1/3); with clip w = (1, 2, 4) the weights b_i/w_i
    are (1/3, 1/6, 1/12), so b' = (4/7, 2/7, 1/7).  Vertex colours are the
    unit vectors, so the Gouraud colour there is b' itself."""
    W = H = 32
    P = 256 * 8 + 128                     # centre of pixel (8, 8) in 16.8 units
    offs = [(-768, 768), (768, 768), (0, -1536)]   # sum to zero: P is the centroid
    ws = [1.0, 2.0, 4.0]                  # powers of two: every float32 step below is exact
    pos = []
    for (dx, dy), w in zip(offs, ws):
        x_ndc = (P + dx) / (128.0 * W) - 1.0
        y_ndc = 1.0 - (P + dy) / (128.0 * H)
        pos.append([x_ndc * w, y_ndc * w, 0.0, w])
    pos = np.array(pos, np.float32)
    color = np.eye(3, dtype=np.float32)
    s = S.Scene(W, H, pos, np.array([[0, 1, 2]], np.int32), color=color)
    X, Y, _, ok = oracle.vertex_stage(s)
    assert ok.all() and list(X) == [P + d[0] for d in offs] and list(Y) == [P + d[1] for d in offs]
    key, _ = oracle.raster_brute(s)
    assert _ids(key)[8, 8] == 0
    rgb = oracle.shade(s, key, perspective=True)[8, 8, :3]
    assert np.allclose(rgb, [4 / 7, 2 / 7, 1 / 7], atol=1e-15)
    assert np.allclose(oracle.shade(s, key)[8, 8, :3], [1 / 3, 1 / 3, 1 / 3], atol=1e-15)


def test_perspective_gouraud_gradient_closed_form():
    """With g = 1 on every channel, dL/dc_v sums v's perspective-correct
    weight over its pixels; the weights at a pixel sum to one, so the total
    is 3 x the covered pixels, as in screen space (an unnormalised weight
    would break it)."""
    sph, mvps = S.sphere_views(num_views=1, width=40, height=40, slices=10, stacks=8, seed=12)
    sph.shade_mode = S.SHADE_GOURAUD
    key, _ = oracle.raster_brute(sph, mvp=mvps[0])
    g = np.zeros((40, 40, 4))
    g[..., :3] = 1.0
    dc, _, _ = oracle.backward(sph, key, g, mvp=mvps[0], perspective=True)
    covered = int((key != EMPTY).sum())
    assert covered > 300
    assert np.isclose(dc.sum(), 3 * covered, rtol=1e-12)
