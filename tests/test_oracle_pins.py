"""Pins of the CPU oracle against closed forms, invariants, a separately
written scanline rasterizer and library routines (no GPU needed).

Every fixed-point convention the oracle follows is a reading (the paper is
silent on rasterization bits); these tests make a plausible slip in any of
them -- a wrong sign, a swapped index, an off-by-one in the fill rule, a
dropped term in the depth -- fail somewhere.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1404_6293_gb300 import scenes as S

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- helpers
def fixed_scene(W, H, verts, tris, zndc=None, color=None, normal=None, mode=0, light=None):
    """Scene whose vertices land exactly on the given 16.8 coordinates.

    With W and H powers of two, x_ndc = X/(128 W) - 1 and y_ndc = 1 - Y/(128 H)
    are exact in float32 and the viewport maps them back to X and Y exactly."""
    assert W & (W - 1) == 0 and H & (H - 1) == 0
    verts = np.asarray(verts, dtype=np.float64)
    n = verts.shape[0]
    x = verts[:, 0] / (128.0 * W) - 1.0
    y = 1.0 - verts[:, 1] / (128.0 * H)
    z = np.zeros(n) if zndc is None else np.asarray(zndc, dtype=np.float64)
    pos = np.stack([x, y, z, np.ones(n)], 1).astype(np.float32)
    assert np.all(pos[:, 0].astype(np.float64) == x) and np.all(pos[:, 1].astype(np.float64) == y)
    return S.Scene(W, H, pos, np.asarray(tris, np.int32).reshape(-1, 3),
                   color=None if color is None else np.asarray(color, np.float32),
                   normal=None if normal is None else np.asarray(normal, np.float32),
                   light_dir=None if light is None else np.asarray(light, np.float32), shade_mode=mode)


def centre(p):
    return 256 * p + 128


def ids(key):
    out = (key & np.uint64(0xFFFFFFFF)).astype(np.int64)
    out[key == EMPTY] = -1
    return out


def depth(key):
    return (key >> np.uint64(32)).astype(np.int64)


# ------------------------------------------------------------ O1-O5 vertex
def test_vertex_stage_corners_and_depth_range():
    W, H = 64, 32
    pos = np.array([[-1, 1, -1, 1], [1, -1, 1, 1], [0, 0, 0, 1], [-1, 1, -0.5, 1], [0, 0, 0.5, 1]],
                   np.float32)
    s = S.Scene(W, H, pos, np.zeros((0, 3), np.int32))
    X, Y, Z, ok = oracle.vertex_stage(s)
    assert ok.tolist() == [1] * 5
    assert (X[0], Y[0], Z[0]) == (0, 0, 0)                      # top-left corner, near plane
    assert (X[1], Y[1], Z[1]) == (256 * W, 256 * H, 16777215)  # bottom-right corner, far plane
    # ndc z = 0: 0.5 * 16777215 = 8388607.5 exactly in float32 -> ties to even
    assert (X[2], Y[2], Z[2]) == (128 * W, 128 * H, 8388608)
    assert Z[3] == 4194304   # 0.25 * 16777215 = 4194303.75 -> 4194304
    assert Z[4] == 12582911  # 0.75 * 16777215 rounds to 12582911.0 in float32


def test_vertex_stage_snap_ties_to_even():
    # x such that sx*256 lands exactly on k + 0.5: W = 1, X/256 = sx, sx*256 = X
    W, H = 1, 1
    xs = [(k + 0.5) / 256.0 for k in (0, 1, 2, 3, 100, 101)]
    pos = np.array([[2 * x - 1, 0, 0, 1] for x in xs], np.float32)
    s = S.Scene(W, H, pos, np.zeros((0, 3), np.int32))
    X, _, _, ok = oracle.vertex_stage(s)
    assert ok.all()
    assert X.tolist() == [0, 2, 2, 4, 100, 102]


def test_vertex_stage_culls():
    W, H = 16, 16
    pos = np.array([
        [0, 0, 0, 0],          # w = 0
        [0, 0, 0, -1],         # w < 0
        [np.nan, 0, 0, 1],     # NaN coordinate -> guard band test fails
        [0, 0, 1.5, 1],        # z beyond far
        [0, 0, -1.0001, 1],    # z before near
        [0, 0, np.nan, 1],     # NaN depth
        [4096.0, 0, 0, 1],     # sx*256 = 2^23 + ... outside the guard band
        [0, 0, 0, 1],          # fine
    ], np.float32)
    s = S.Scene(W, H, pos, np.zeros((0, 3), np.int32))
    _, _, _, ok = oracle.vertex_stage(s)
    assert ok.tolist() == [0, 0, 0, 0, 0, 0, 0, 1]


def test_guard_band_limit_is_2_pow_23():
    # W = 256: sx*256 = (x*0.5+0.5)*65536; |fx| < 2^23 <=> (x*0.5+0.5) < 128
    W = 256
    inside = 2 * (127.99 - 0.5)
    outside = 2 * (128.0 - 0.5)
    pos = np.array([[inside, 0, 0, 1], [outside, 0, 0, 1]], np.float32)
    _, _, _, ok = oracle.vertex_stage(S.Scene(W, W, pos, np.zeros((0, 3), np.int32)))
    assert ok.tolist() == [1, 0]


def test_mvp_identity_equals_none_and_scaling_matrix():
    s = S.random_triangles(64, 64, 50, 10.0, seed=7)
    ident = np.eye(4, dtype=np.float32).ravel()
    a = oracle.vertex_stage(s)
    b = oracle.vertex_stage(s, mvp=ident)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    # w scaled by 2 with xyz scaled by 2: the projective divide undoes it exactly
    M = (2 * np.eye(4)).astype(np.float32).ravel()
    c = oracle.vertex_stage(s, mvp=M)
    for u, v in zip(a, c):
        assert np.array_equal(u, v)


def test_mvp_row_major_translation():
    # row-major M with a translation in the last column moves x by +0.5 NDC
    M = np.eye(4, dtype=np.float32)
    M[0, 3] = 0.5
    pos = np.array([[-1, 1, 0, 1]], np.float32)
    X, Y, _, ok = oracle.vertex_stage(S.Scene(64, 64, pos, np.zeros((0, 3), np.int32)), mvp=M.ravel())
    assert ok[0] == 1 and X[0] == 256 * 64 // 4 and Y[0] == 0


# --------------------------------------------------------- coverage pins
@pytest.mark.parametrize("W,H", [(8, 8), (16, 8), (32, 64), (64, 64)])
@pytest.mark.parametrize("diag", [0, 1])
@pytest.mark.parametrize("flip", [0, 1])
def test_full_screen_quad_covers_every_pixel_once(W, H, diag, flip):
    X1, Y1 = 256 * W, 256 * H
    v = [(0, 0), (X1, 0), (X1, Y1), (0, Y1)]
    t = [(0, 1, 2), (0, 2, 3)] if diag == 0 else [(0, 1, 3), (1, 2, 3)]
    if flip:
        t = [(a, c, b) for (a, b, c) in t]
    s = fixed_scene(W, H, v, t, zndc=[0.1, -0.2, 0.3, 0.0])
    key, cnt, st = oracle.raster_brute(s, with_count=True)
    assert st == 0
    assert (cnt == 1).all()
    assert (key != EMPTY).all()


def _grid_scene(W, H, x0, y0, nx, ny, cell, jitter, seed, centre_snap=False):
    rng = np.random.default_rng(seed)
    verts = []
    for j in range(ny + 1):
        for i in range(nx + 1):
            X = x0 + i * cell
            Y = y0 + j * cell
            if 0 < i < nx and 0 < j < ny:
                if centre_snap and rng.random() < 0.5:
                    X = 256 * (X // 256) + 128
                    Y = 256 * (Y // 256) + 128
                else:
                    X += int(rng.integers(-jitter, jitter + 1))
                    Y += int(rng.integers(-jitter, jitter + 1))
            verts.append((X, Y))
    tris = []
    for j in range(ny):
        for i in range(nx):
            a = j * (nx + 1) + i
            b, c, d = a + 1, a + nx + 1, a + nx + 2
            if rng.random() < 0.5:
                tris += [(a, b, d), (a, d, c)]
            else:
                tris += [(a, b, c), (b, d, c)]
            if rng.random() < 0.5:  # random input winding
                tris[-1] = (tris[-1][0], tris[-1][2], tris[-1][1])
    z = rng.uniform(-0.9, 0.9, len(verts))
    return fixed_scene(W, H, verts, tris, zndc=z)


@pytest.mark.parametrize("seed", range(6))
def test_watertight_grid_interior_once_exterior_never(seed):
    W = H = 64
    rng = np.random.default_rng(100 + seed)
    cell = int(rng.integers(600, 1500))
    x0 = int(rng.integers(0, 2000))
    y0 = int(rng.integers(0, 2000))
    if seed % 2 == 0:  # boundary through pixel centres
        x0 = centre(x0 // 256)
        y0 = centre(y0 // 256)
    nx = (256 * W - x0 - 300) // cell
    ny = (256 * H - y0 - 300) // cell
    s = _grid_scene(W, H, x0, y0, nx, ny, cell, cell // 4, seed, centre_snap=(seed >= 3))
    _, cnt, st = oracle.raster_brute(s, with_count=True)
    assert st == 0
    x1, y1 = x0 + nx * cell, y0 + ny * cell
    P = centre(np.arange(W))
    Q = centre(np.arange(H))
    inside = ((P[None, :] >= x0) & (P[None, :] < x1)) & ((Q[:, None] >= y0) & (Q[:, None] < y1))
    assert np.array_equal(cnt, inside.astype(np.uint32))


@pytest.mark.parametrize("L", [1, 2, 3, 7, 12])
def test_right_triangle_lattice_count_and_depth(L):
    # legs along the top and left edges starting at a pixel centre: covered
    # centres are (i, j) >= 0 with i + j < L, so L(L+1)/2 of them; b1 = i/L,
    # b2 = j/L there, so z = floor(Z0 + (i (Z1-Z0) + j (Z2-Z0)) / L).
    W = H = 32
    a, b = 3, 5
    v0 = (centre(a), centre(b))
    v = [v0, (v0[0] + 256 * L, v0[1]), (v0[0], v0[1] + 256 * L)]
    s = fixed_scene(W, H, v, [(0, 1, 2)], zndc=[-0.5, 0.5, 0.0])
    key, cnt, st = oracle.raster_brute(s, with_count=True)
    assert cnt.sum() == L * (L + 1) // 2
    _, _, Z, _ = oracle.vertex_stage(s)
    Z0, Z1, Z2 = (int(z) for z in Z)
    for j in range(L):
        for i in range(L - j):
            k = key[b + j, a + i]
            assert ids(np.array([k]))[0] == 0
            num = Z0 * L + i * (Z1 - Z0) + j * (Z2 - Z0)
            assert depth(np.array([k]))[0] == num // L  # python // is floor
    assert (cnt[b, a:a + L] == 1).all() and (cnt[b:b + L, a] == 1).all()
    # the vertex sits on a covered pixel centre: depth there is exactly Z0
    assert depth(np.array([key[b, a]]))[0] == Z0


def test_top_left_rule_example_orientation():
    # v0=(0,0), v1=(1,0), v2=(0,1) in pixel steps: edge 0->1 is a top edge,
    # 2->0 a left edge, 1->2 neither.  Centres on the top and left edges are
    # covered; the centre on the hypotenuse is not.
    W = H = 16
    c = (centre(4), centre(4))
    v = [c, (c[0] + 512, c[1]), (c[0], c[1] + 512)]
    key, cnt, _ = oracle.raster_brute(fixed_scene(W, H, v, [(0, 1, 2)]), with_count=True)
    assert cnt[4, 4] == 1 and cnt[4, 5] == 1 and cnt[5, 4] == 1   # on top / left edges
    assert cnt[4, 6] == 0 and cnt[6, 4] == 0 and cnt[5, 5] == 0   # right vertex, bottom vertex, hypotenuse
    # mirrored triangle: hypotenuse on the top-left side, legs bottom/right
    v = [(c[0] + 512, c[1] + 512), (c[0], c[1] + 512), (c[0] + 512, c[1])]
    _, cnt2, _ = oracle.raster_brute(fixed_scene(W, H, v, [(0, 1, 2)]), with_count=True)
    assert cnt2[5, 5] == 1                     # on the (top-left) hypotenuse
    assert cnt2[6, 6] == 0 and cnt2[6, 5] == 0 and cnt2[5, 6] == 0  # bottom/right legs excluded


def test_one_pixel_square_through_centres_covers_exactly_one():
    W = H = 16
    for a, b in [(0, 0), (7, 3), (14, 14)]:
        x0, y0 = centre(a), centre(b)
        v = [(x0, y0), (x0 + 256, y0), (x0 + 256, y0 + 256), (x0, y0 + 256)]
        _, cnt, _ = oracle.raster_brute(fixed_scene(W, H, v, [(0, 1, 2), (0, 2, 3)]), with_count=True)
        assert cnt.sum() == 1 and cnt[b, a] == 1


def test_degenerate_and_subpixel_triangles():
    W = H = 16
    c = centre(5)
    v = [(c, c), (c + 512, c), (c + 1024, c),          # collinear: A = 0
         (c + 10, c + 10), (c + 60, c + 10), (c + 10, c + 60)]  # no centre inside
    _, cnt, st = oracle.raster_brute(fixed_scene(W, H, v, [(0, 1, 2), (3, 4, 5)]), with_count=True)
    assert st == 0 and cnt.sum() == 0


def test_golden_hand_derived_4x4():
    with open(os.path.join(GOLDEN, "quad_4x4.json")) as f:
        g = json.load(f)
    s = fixed_scene(4, 4, g["verts_fixed"], g["tris"], zndc=g["zndc"])
    key, st = oracle.raster_brute(s)
    assert st == 0
    assert ids(key).tolist() == g["expected_id"]
    assert depth(key).tolist() == g["expected_depth"]


# ------------------------------------------------------------ ties (O10)
def test_identical_triangles_lower_index_wins():
    s = S.random_triangles(64, 64, 40, 12.0, seed=3)
    t = np.concatenate([s.tris[5:6], s.tris, s.tris[5:6]])
    s2 = S.Scene(s.width, s.height, s.pos, t)
    key, _ = oracle.raster_brute(s2)
    k1, _ = oracle.raster_brute(S.Scene(s.width, s.height, s.pos, s.tris[5:6]))
    cov = k1 != EMPTY
    i = ids(key)
    # triangle 0 (a copy of tris[5]) beats the later copies at every pixel where tris[5] wins
    base, _ = oracle.raster_brute(s)
    won = ids(base) == 5
    assert (i[won] == 0).all()
    assert (i[cov] != 6).all() and (i[cov] != 41).all()


def test_coplanar_overlap_takes_min_index():
    W = H = 16
    v = [(0, 0), (4096, 0), (0, 4096), (4096, 4096)]
    s = fixed_scene(W, H, v, [(1, 3, 2), (0, 1, 2), (0, 1, 3)], zndc=[0.25] * 4)
    key, cnt, _ = oracle.raster_brute(s, with_count=True)
    i = ids(key)
    d = depth(key)
    assert len(set(d[key != EMPTY].tolist())) == 1
    # each pixel goes to the lowest-numbered triangle covering it
    for t in range(3):
        alone, _ = oracle.raster_brute(S.Scene(W, H, s.pos, s.tris[t:t + 1]))
        lower = np.zeros_like(alone, dtype=bool)
        for u in range(t):
            au, _ = oracle.raster_brute(S.Scene(W, H, s.pos, s.tris[u:u + 1]))
            lower |= au != EMPTY
        assert ((i == t) == ((alone != EMPTY) & ~lower)).all()


# ------------------------------------------------------- depth (O9) pins
def test_constant_depth_and_range():
    s = S.random_triangles(64, 64, 60, 15.0, seed=11)
    key, _ = oracle.raster_brute(s)
    _, _, Z, ok = oracle.vertex_stage(s)
    i = ids(key)
    d = depth(key)
    for t in np.unique(i[i >= 0]):
        z3 = Z[s.tris[t]].astype(np.int64)
        sel = i == t
        assert d[sel].min() >= z3.min() and d[sel].max() <= z3.max()
    # flat triangles: all three depths equal -> z is that depth exactly
    pos = s.pos.copy()
    pos[:, 2] = 0.0
    key2, _ = oracle.raster_brute(S.Scene(64, 64, pos, s.tris))
    assert (depth(key2)[key2 != EMPTY] == 8388608).all()


# --------------------------------------------------- independent cross-checks
def _tiny_scene(seed):
    rng = np.random.default_rng(seed)
    W = int(rng.integers(1, 65))
    H = int(rng.integers(1, 65))
    T = int(rng.integers(0, 51))
    V = 3 * T + int(rng.integers(0, 4))
    pos = np.empty((V, 4), np.float32)
    pos[:, :2] = rng.uniform(-1.3, 1.3, (V, 2))
    if rng.random() < 0.3:  # snap some vertices to pixel centres / edges for exact ties
        k = rng.random(V) < 0.5
        pos[k, 0] = ((rng.integers(0, 2 * W + 1, k.sum()) / (2.0 * W)) * 2 - 1)
        pos[k, 1] = ((rng.integers(0, 2 * H + 1, k.sum()) / (2.0 * H)) * 2 - 1)
    pos[:, 2] = rng.uniform(-1.05, 1.05, V)
    pos[:, 3] = rng.choice([1.0, 1.0, 1.0, 0.5, 2.0, -1.0, 0.0], V)
    pos[:, :3] *= np.where(pos[:, 3:] > 0, pos[:, 3:], 1.0)
    if rng.random() < 0.2:  # shared vertices and duplicates
        tris = rng.integers(0, V, (T, 3)) if V else np.zeros((0, 3))
    else:
        tris = np.arange(3 * T).reshape(T, 3)
    return S.Scene(W, H, pos, np.asarray(tris, np.int32))


def test_scanline_matches_brute_force_on_tiny_scenes():
    n = int(os.environ.get("PIKO_TINY_SCENES", "600"))
    for seed in range(n):
        s = _tiny_scene(seed)
        kb, st1 = oracle.raster_brute(s)
        ks, st2 = oracle.raster_scanline(s)
        assert st1 == st2 == 0
        assert np.array_equal(kb, ks), f"seed {seed}"


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_bbox_matches_brute_force(threads):
    for seed in range(40):
        s = _tiny_scene(1000 + seed)
        kb, _ = oracle.raster_brute(s)
        kx, _ = oracle.raster_bbox(s, threads=threads)
        assert np.array_equal(kb, kx), f"seed {seed}"
    s = S.random_triangles(256, 256, 1000, 40.0)
    kb, _ = oracle.raster_brute(s)
    kx, _ = oracle.raster_bbox(s, threads=threads)
    assert np.array_equal(kb, kx)


def test_keys_at_matches_full_frame():
    s = S.random_triangles(128, 96, 300, 20.0, seed=5)
    kb, _ = oracle.raster_brute(s)
    rng = np.random.default_rng(0)
    pix = np.stack([rng.integers(0, 128, 500), rng.integers(0, 96, 500)], 1)
    k, _ = oracle.keys_at(s, pix)
    assert np.array_equal(k, kb[pix[:, 1], pix[:, 0]])


def test_bad_index_culls_and_reports():
    s = S.random_triangles(64, 64, 20, 12.0, seed=9)
    t = s.tris.copy()
    t[3] = [0, 1, 10_000]
    t[7] = [-1, 2, 3]
    key, st = oracle.raster_brute(S.Scene(64, 64, s.pos, t))
    assert st == oracle.BAD_INDEX
    keep = np.array([i for i in range(20) if i not in (3, 7)])
    ref, st2 = oracle.raster_brute(S.Scene(64, 64, s.pos, s.tris[keep]))
    assert st2 == 0
    # same coverage and depth; ids map through keep
    assert np.array_equal(key == EMPTY, ref == EMPTY)
    m = ref != EMPTY
    assert np.array_equal(depth(key)[m], depth(ref)[m])
    assert np.array_equal(ids(key)[m], keep[ids(ref)[m]])


# ------------------------------------------------------------ binary16
def test_half_rounding_against_numpy():
    rng = np.random.default_rng(1)
    vals = np.concatenate([
        rng.normal(0, 1, 3000), rng.normal(0, 1e-5, 500), rng.normal(0, 3e4, 500),
        [0.0, -0.0, 1.0, -1.0, 65504.0, 65519.999, 65520.0, 1e6, -1e6, 2.0 ** -24, 2.0 ** -25,
         3 * 2.0 ** -26, 2.0 ** -25 * 1.0000001, 6.097555e-5, 1 + 2 ** -11, 1 + 3 * 2 ** -11,
         2048 + 1, 2048 + 3, 0.1, 1 / 3],
    ])
    for v in vals:
        h = oracle.half_from_double(float(v))
        with np.errstate(over="ignore"):
            ref = int(np.array(v, dtype=np.float64).astype(np.float16).view(np.uint16))
            hv = float(np.float16(v))
        assert h == ref, (v, hex(h), hex(ref))
        if not math.isinf(hv):
            assert oracle.double_from_half(h) == float(np.float16(v))
    assert oracle.half_from_double(float("nan")) & 0x7C00 == 0x7C00


def test_half_ties_to_even_explicit():
    # 1 + 2^-11 is halfway between 1 and 1 + 2^-10: ties to the even mantissa (1.0)
    assert oracle.half_from_double(1 + 2 ** -11) == 0x3C00
    assert oracle.half_from_double(1 + 3 * 2 ** -11) == 0x3C02
    assert oracle.half_from_double(2.0 ** -25) == 0x0000      # halfway to the smallest subnormal
    assert oracle.half_from_double(3 * 2.0 ** -25) == 0x0002  # 1.5 quanta -> 2
    assert oracle.half_from_double(65520.0) == 0x7C00         # overflow to infinity
    assert oracle.half_from_double(65504.0) == 0x7BFF


# ------------------------------------------------------------- shading O11
def test_listing1_constants_golden():
    with open(os.path.join(GOLDEN, "listing1_shading.json")) as f:
        g = json.load(f)
    W = H = 16
    v = [(0, 0), (4096, 0), (0, 4096), (4096, 4096)]
    L = np.array(g["light_unnormalised"], np.float64)
    L = (L / np.linalg.norm(L)).astype(np.float32)
    nrm = np.tile(L, (4, 1))  # every normal along the light
    s = fixed_scene(W, H, v, [(0, 1, 2), (1, 3, 2)], normal=nrm, mode=1, light=L)
    key, _ = oracle.raster_brute(s)
    rgba = oracle.shade(s, key)
    assert np.allclose(rgba[..., :3], np.array(g["material"]), atol=1e-6)
    assert (rgba[..., 3] == 1.0).all()
    # normals opposite the light: clamped to zero, or -material unclamped
    s.normal = -nrm
    assert np.allclose(oracle.shade(s, key)[..., :3], 0.0)
    assert np.allclose(oracle.shade(s, key, unclamped=True)[..., :3], -np.array(g["material"]), atol=1e-6)


def test_gouraud_constant_colour_and_vertex_value():
    s = S.random_triangles(64, 64, 80, 15.0, seed=13)
    s.color = np.tile(np.array([[0.25, 0.5, 0.75]], np.float32), (s.num_vertices, 1))
    key, _ = oracle.raster_brute(s)
    rgba = oracle.shade(s, key)
    m = key != EMPTY
    assert np.allclose(rgba[m][:, :3], [0.25, 0.5, 0.75], atol=1e-12)
    assert (rgba[~m] == 0).all() and (rgba[m][:, 3] == 1).all()
    # at a vertex sitting on a covered pixel centre, the colour is that vertex's
    # (both edges meeting at v0 run upward, so both are top-left and v0 is covered)
    c = (centre(3), centre(4))
    v = [c, (c[0] + 2048, c[1] - 300), (c[0] + 100, c[1] + 1900)]
    col = np.array([[0.1, 0.2, 0.3], [0.9, 0.8, 0.7], [0.5, 0.5, 0.5]], np.float32)
    s2 = fixed_scene(32, 32, v, [(0, 1, 2)], color=col, mode=0)
    key2, _ = oracle.raster_brute(s2)
    assert ids(key2)[4, 3] == 0
    assert np.allclose(oracle.shade(s2, key2)[4, 3, :3], col[0].astype(np.float64), atol=0)


def test_gouraud_is_affine_in_screen_space():
    # along a row inside a triangle, colour steps by a constant per pixel
    c = (centre(2), centre(2))
    v = [c, (c[0] + 256 * 20, c[1]), (c[0], c[1] + 256 * 20)]
    col = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    s = fixed_scene(32, 32, v, [(0, 1, 2)], color=col, mode=0)
    key, _ = oracle.raster_brute(s)
    rgba = oracle.shade(s, key)
    row = rgba[2, 2:20, 0]
    assert np.allclose(np.diff(row), 1.0 / 20.0, atol=1e-12)
    col_g = rgba[2:20, 2, 1]
    assert np.allclose(np.diff(col_g), 1.0 / 20.0, atol=1e-12)


# ---------------------------------------------------------- light pass O12
def test_light_pass_closed_forms():
    W, H = 8, 4
    D = 8.0
    r2 = (D / 4) ** 2
    key = np.full((H, W), EMPTY, np.uint64)
    key[1, 2] = np.uint64(8388608) << np.uint64(32)  # depth z -> S.z = z/16777215 * D
    n = np.zeros((H, W, 4), np.float16)
    n[1, 2, :3] = [0, 0, -1]
    a = np.zeros((H, W, 4), np.float16)
    a[1, 2, :3] = [0.5, 0.25, 1.0]
    Sz = 8388608 / 16777215 * D
    d = 3.0
    lights = np.array([[2.5, 1.5, Sz - d, 0.75],     # straight along the normal
                       [2.5, 1.5, Sz + d, 0.5]],     # behind the surface: no light
                      np.float32)
    out = oracle.light_pass(key, n.view(np.uint16), a.view(np.uint16), lights)
    term = 0.75 * 1.0 / (1.0 + d * d / r2)
    assert np.allclose(out[1, 2, :3], np.array([0.5, 0.25, 1.0]) * term, rtol=1e-6)
    assert out[1, 2, 3] == 1.0
    m = key == EMPTY
    assert (out[m] == 0).all()


# ------------------------------------------------------------ gradients O13
def _fd_scene():
    s = S.random_triangles(48, 48, 90, 10.0, seed=21, shade_mode=S.SHADE_LAMBERT, with_normals=True)
    s.light_dir = np.array([0.3, -0.4, -0.866], np.float32)
    return s


def test_backward_matches_central_differences():
    s = _fd_scene()
    key, _ = oracle.raster_brute(s)
    tgt = S.target_image(48, 48, seed=3)[0]
    rgba = oracle.shade(s, key)
    g = np.zeros((48, 48, 4))
    g[..., :3] = 2.0 * (rgba[..., :3] - tgt[..., :3])
    dc, dn, dl = oracle.backward(s, key, g)
    col = s.color.astype(np.float64)
    nrm = s.normal.astype(np.float64)
    L = s.light_dir.astype(np.float64)

    def fd(which, idx):
        c, n, l = col.copy(), nrm.copy(), L.copy()
        arr = {"c": c, "n": n, "l": l}[which]
        th = arr.flat[idx]
        h = 1e-6 * max(1.0, abs(th))
        arr.flat[idx] = th + h
        lp = oracle.loss(s, key, tgt, color=c, normal=n, light=l)
        arr.flat[idx] = th - h
        lm = oracle.loss(s, key, tgt, color=c, normal=n, light=l)
        return (lp - lm) / (2 * h)

    # 128 seeded (vertex, channel) indices per array and the 3 light components:
    # 259 parameters, each against a float64 central difference of the loss
    rng = np.random.default_rng(0)
    used = np.unique(s.tris[np.unique(ids(key)[key != EMPTY])])
    params = np.array([3 * v + ch for v in used for ch in range(3)])
    assert params.size >= 128
    for which, an in (("c", dc), ("n", dn)):
        scale = np.abs(an).max()
        assert scale > 0
        for idx in rng.choice(params, 128, replace=False):
            v, ch = divmod(int(idx), 3)
            num = fd(which, int(idx))
            assert abs(num - an[v, ch]) <= 1e-4 * max(abs(an[v, ch]), 1e-3 * scale) + 1e-9
    for ch in range(3):
        num = fd("l", ch)
        assert abs(num - dl[ch]) <= 1e-4 * max(abs(dl[ch]), 1e-3 * np.abs(dl).max())


def test_gouraud_gradient_closed_form():
    s = S.random_triangles(32, 32, 20, 10.0, seed=22)
    key, _ = oracle.raster_brute(s)
    g = np.zeros((32, 32, 4))
    g[..., :3] = 1.0
    dc, _, _ = oracle.backward(s, key, g)
    # with g = 1, dL/dc_v sums the barycentric weight of v over its pixels,
    # and the weights at a pixel sum to one: total = 3 * covered pixels
    assert np.isclose(dc.sum(), 3 * (key != EMPTY).sum(), rtol=1e-12)


# ---------------------------------------------------------- generators
def test_splitmix64_reference_outputs():
    # first outputs of SplitMix64 seeded with 0 (Steele et al. 2014 reference code)
    r = S.SplitMix64(0).next_u64(3)
    assert [int(x) for x in r] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_random_triangle_generator_statistics():
    s = S.random_triangles()
    assert s.num_triangles == 1000 and s.num_vertices == 3000
    X, Y, Z, ok = oracle.vertex_stage(s)
    t = s.tris
    A = ((X[t[:, 1]] - X[t[:, 0]]).astype(np.float64) * (Y[t[:, 2]] - Y[t[:, 0]]) -
         (X[t[:, 2]] - X[t[:, 0]]).astype(np.float64) * (Y[t[:, 1]] - Y[t[:, 0]]))
    area = np.abs(A) / 2 / 65536
    # expected triangle area for vertices uniform in a disc of radius R is 35 R^2 / (48 pi)
    assert abs(area.mean() / (35 * 40 ** 2 / (48 * np.pi)) - 1) < 0.1


def test_heightfield_generator_area_band():
    s = S.heightfield()
    assert s.num_triangles == 1_000_000 and s.num_vertices == 501_501
    X, Y, Z, ok = oracle.vertex_stage(s)
    assert ok.all()
    t = s.tris
    A = ((X[t[:, 1]] - X[t[:, 0]]).astype(np.float64) * (Y[t[:, 2]] - Y[t[:, 0]]) -
         (X[t[:, 2]] - X[t[:, 0]]).astype(np.float64) * (Y[t[:, 1]] - Y[t[:, 0]]))
    area = np.abs(A) / 2 / 65536
    cx = (X[t].mean(1) / 256)
    cy = (Y[t].mean(1) / 256)
    on = (cx >= 0) & (cx < 1920) & (cy >= 0) & (cy < 1080)
    p5, p95 = np.percentile(area[on], [5, 95])
    assert 2.0 <= p5 and p95 <= 10.0
    assert area[on].sum() > 0.99 * 1920 * 1080  # the grid fills the screen


def test_power_law_and_sphere_generators():
    s = S.power_law_triangles(num_tris=20000)
    X, Y, _, ok = oracle.vertex_stage(s)
    assert ok.all()
    t = s.tris
    A = ((X[t[:, 1]] - X[t[:, 0]]).astype(np.float64) * (Y[t[:, 2]] - Y[t[:, 0]]) -
         (X[t[:, 2]] - X[t[:, 0]]).astype(np.float64) * (Y[t[:, 1]] - Y[t[:, 0]]))
    area = np.abs(A) / 2 / 65536
    # pdf ~ a^-2 on [1, amax]: median = 2 / (1 + 1/amax) ~ 2, mean = ln(amax) / (1 - 1/amax)
    assert abs(np.median(area) - 2.0) < 0.15
    sph, mvps = S.sphere_views(num_views=4)
    assert sph.num_vertices == 199 * 250 + 2 and sph.num_triangles == 99_500
    assert mvps.shape == (4, 16)


# ------------------------------------------------- O12 G-buffer layout, O13 loss
def test_gbuffer_words_hand_derived_4x4():
    """G-buffer output layout (normal + 0, albedo + alpha 1, empty pixels all
    zero) and binary16 words against values derived by hand."""
    with open(os.path.join(GOLDEN, "gbuffer_4x4.json")) as f:
        g = json.load(f)
    s = fixed_scene(4, 4, g["verts_fixed"], g["tris"], color=g["albedo"], normal=g["normal"], mode=2)
    key, st = oracle.raster_brute(s)
    assert st == 0
    gn, ga = oracle.shade(s, key)
    assert gn.dtype == np.uint16 and ga.dtype == np.uint16 and gn.shape == (4, 4, 4)
    for j in range(4):
        for i in range(4):
            k = f"{i},{j}"
            if k in g["normal_words"]:
                assert gn[j, i].tolist() == g["normal_words"][k], k
                assert ga[j, i].tolist() == g["albedo_words"][k], k
            else:
                assert key[j, i] == EMPTY, k
                assert gn[j, i].tolist() == [0, 0, 0, 0] and ga[j, i].tolist() == [0, 0, 0, 0], k


def _loss_scene(mode, color, normal=None, light=None):
    with open(os.path.join(GOLDEN, "gbuffer_4x4.json")) as f:
        g = json.load(f)
    return fixed_scene(4, 4, g["verts_fixed"], g["tris"], color=color, normal=normal, mode=mode, light=light)


def test_loss_closed_form_gouraud_one_triangle():
    """One constant-colour triangle over six of 16 pixels: covered pixels
    contribute |c - t|^2, empty ones |t|^2 over RGB; alpha never enters."""
    c = np.array([0.5, 0.25, 1.0])
    s = _loss_scene(0, np.tile(c, (4, 1)))
    key, st = oracle.raster_brute(s)
    assert st == 0 and int((key != EMPTY).sum()) == 6
    target = np.zeros((4, 4, 4), np.float32)
    target[..., 3] = 5.0                       # alpha of the target is ignored
    target[key == EMPTY, :3] = 0.5             # empty pixels: rgb 0 against 0.5
    # 6 * (0.25 + 0.0625 + 1) + 10 * 3 * 0.25 = 7.875 + 7.5
    assert oracle.loss(s, key, target) == 15.375
    target[key != EMPTY, :3] = c                # covered pixels exact: only the empty ones remain
    assert oracle.loss(s, key, target) == 7.5


def test_loss_closed_form_lambert_clamp():
    """Lambert with n = (0, 0, 1), albedo R linear in x (0.125 + 0.25 i at
    column i): L = (0, 0, 0.5) gives sum over covered (i, j) of
    (0.5 (0.125 + 0.25 i))^2 = 0.25 (3 * 0.125^2 + 2 * 0.375^2 + 0.625^2) =
    0.1796875; L = (0, 0, -0.5) clamps to 0 (loss 0) unless unclamped."""
    col = np.array([[0.0, 0, 0], [1.0, 0, 0], [0, 0, 0], [0.0, 0, 0]])
    nrm = np.tile([0.0, 0.0, 1.0], (4, 1))
    target = np.zeros((4, 4, 4), np.float32)
    s = _loss_scene(1, col, nrm, [0.0, 0.0, 0.5])
    key, _ = oracle.raster_brute(s)
    assert oracle.loss(s, key, target) == 0.1796875
    s = _loss_scene(1, col, nrm, [0.0, 0.0, -0.5])
    assert oracle.loss(s, key, target) == 0.0
    assert oracle.loss(s, key, target, unclamped=True) == 0.1796875
