"""Seeded synthetic scene generators: the inputs of the rasterizer, nothing else.

This module produces triangle lists with per-vertex attributes (the input a
raster pipeline consumes, Sec. 4.1 and Sec. 7.1 of the Piko paper) and holds
none of the rasterizer's own arithmetic: no transform, snapping, coverage,
depth or shading happens here.  Both the CUDA path and the CPU oracle take
their inputs from these functions, so that neither feeds the other.

Randomness comes from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: output i of a stream is the SplitMix64 finaliser applied to
``base + (i + 1) * 0x9E3779B97F4A7C15``.

The paper's own test scenes (Sec. 7.2, Fig. "rastpics") are not available;
the generators below stand in for them with the shapes the paper describes:
many small triangles, a mix of small and large ones, and so on.

Shading modes (the ``shade_mode`` field of a scene):
  0 Gouraud   interpolated per-vertex colour
  1 Lambert   colour times max(0, n . L), after Listing 1 of the paper
  2 G-buffer  depth|ID plus FP16 normal and albedo, for a deferred light pass
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

SHADE_GOURAUD = 0
SHADE_LAMBERT = 1
SHADE_GBUFFER = 2

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class SplitMix64:
    """Counter-based SplitMix64 stream: draws are a pure function of (seed, counter)."""

    def __init__(self, seed: int):
        self.base = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.counter = 0

    def next_u64(self, n: int) -> np.ndarray:
        idx = np.arange(self.counter + 1, self.counter + n + 1, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            return _mix64(self.base + idx * _GAMMA)

    def uniform(self, n: int) -> np.ndarray:
        """Float64 in [0, 1) from the top 53 bits."""
        return (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def integers(self, lo: int, hi: int, n: int) -> np.ndarray:
        """Integers in [lo, hi) (hi - lo well below 2**53)."""
        return lo + np.floor(self.uniform(n) * (hi - lo)).astype(np.int64)


@dataclass
class Scene:
    """One scene: a triangle list with per-vertex attributes and a framebuffer size.

    pos        float32 [V,4]  homogeneous vertex positions (x, y, z, w)
    tris       int32   [T,3]  vertex indices
    color      float32 [V,3]  per-vertex RGB (None: constant material)
    normal     float32 [V,3]  per-vertex normals (Lambert / G-buffer)
    mvp        float32 [16]   row-major 4x4 applied to pos (None: identity)
    light_dir  float32 [3]    directional light, used as given (Lambert)
    """

    width: int
    height: int
    pos: np.ndarray
    tris: np.ndarray
    color: Optional[np.ndarray] = None
    normal: Optional[np.ndarray] = None
    mvp: Optional[np.ndarray] = None
    light_dir: Optional[np.ndarray] = None
    shade_mode: int = SHADE_GOURAUD
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def num_vertices(self) -> int:
        return int(self.pos.shape[0])

    @property
    def num_triangles(self) -> int:
        return int(self.tris.shape[0])


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def listing1_light() -> np.ndarray:
    """The light vector of Listing 1, normalize(1,1,1), rounded to float32."""
    return _f32(np.full(3, 1.0 / np.sqrt(3.0)))


# --------------------------------------------------------------------------
# Random small triangles (256x256, 1,000 triangles, 40-px radius)
# --------------------------------------------------------------------------
def random_triangles(width=256, height=256, num_tris=1000, radius_px=40.0, seed=1235,
                     shade_mode=SHADE_GOURAUD, with_normals=False) -> Scene:
    """Independent triangles: a uniform centre in NDC [-1,1]^2, each vertex
    within ``radius_px`` pixels of it (uniform over the disc), a uniform
    24-bit depth per vertex expressed as NDC z, and uniform RGB in [0,1]."""
    rng = SplitMix64(seed)
    T = int(num_tris)
    c = rng.uniform(2 * T).reshape(T, 2) * 2.0 - 1.0
    r = radius_px * np.sqrt(rng.uniform(3 * T)).reshape(T, 3)
    th = rng.uniform(3 * T).reshape(T, 3) * (2.0 * np.pi)
    x = c[:, :1] + r * np.cos(th) * (2.0 / width)
    y = c[:, 1:] + r * np.sin(th) * (2.0 / height)
    zint = rng.integers(0, 1 << 24, 3 * T).reshape(T, 3)
    z = 2.0 * zint / 16777215.0 - 1.0
    pos = np.stack([x, y, z, np.ones_like(x)], axis=-1).reshape(3 * T, 4)
    color = rng.uniform(9 * T).reshape(3 * T, 3)
    normal = None
    if with_normals or shade_mode != SHADE_GOURAUD:
        v = rng.uniform(9 * T).reshape(3 * T, 3) * 2.0 - 1.0
        v[:, 2] = -np.abs(v[:, 2]) - 0.25
        normal = v / np.linalg.norm(v, axis=1, keepdims=True)
    return Scene(width, height, _f32(pos), _i32(np.arange(3 * T).reshape(T, 3)),
                 color=_f32(color), normal=None if normal is None else _f32(normal),
                 light_dir=listing1_light() if shade_mode == SHADE_LAMBERT else None,
                 shade_mode=shade_mode, name=f"random{T}_{width}x{height}")


# --------------------------------------------------------------------------
# Displaced heightfield grid (1920x1080, 1000x500 quads -> 1M triangles)
# --------------------------------------------------------------------------
def _look_at_perspective(eye, target, up, fovy_deg, aspect, near, far) -> np.ndarray:
    """Row-major 4x4 projection * view (OpenGL conventions), float64."""
    eye, target, up = (np.asarray(v, dtype=np.float64) for v in (eye, target, up))
    f = target - eye
    f /= np.linalg.norm(f)
    s = np.cross(f, up)
    s /= np.linalg.norm(s)
    u = np.cross(s, f)
    view = np.eye(4)
    view[0, :3], view[1, :3], view[2, :3] = s, u, -f
    view[:3, 3] = -view[:3, :3] @ eye
    t = 1.0 / np.tan(np.radians(fovy_deg) / 2.0)
    proj = np.zeros((4, 4))
    proj[0, 0] = t / aspect
    proj[1, 1] = t
    proj[2, 2] = (far + near) / (near - far)
    proj[2, 3] = 2.0 * far * near / (near - far)
    proj[3, 2] = -1.0
    return proj @ view


def heightfield(width=1920, height=1080, nx=1000, ny=500, seed=1236,
                shade_mode=SHADE_LAMBERT, with_color=False, overfill=1.15) -> Scene:
    """A grid of nx x ny quads, two triangles each, displaced by a seeded sum
    of 8 sinusoid octaves, seen by a slightly tilted perspective camera that
    the grid overfills.  World-space positions (w = 1) plus an MVP matrix;
    per-vertex normals from central differences of the height samples."""
    rng = SplitMix64(seed)
    aspect = width / height
    sx = aspect
    sz = sx * ny / nx
    gx = np.linspace(-sx, sx, nx + 1)
    gz = np.linspace(-sz, sz, ny + 1)
    X, Z = np.meshgrid(gx, gz)                    # [ny+1, nx+1]
    amp = 0.02 * sx
    hgt = np.zeros_like(X)
    dirs = rng.uniform(8) * 2.0 * np.pi
    phases = rng.uniform(8) * 2.0 * np.pi
    for k in range(8):
        freq = (2.0 ** k) * 1.5 / sx
        d = np.cos(dirs[k]) * X + np.sin(dirs[k]) * Z
        hgt += amp * (0.5 ** k) * np.sin(freq * d + phases[k])
    pos = np.stack([X, hgt, Z, np.ones_like(X)], axis=-1).reshape(-1, 4)
    # normals: n = normalize(-dh/dx, 1, -dh/dz) from central differences
    dhx = np.gradient(hgt, gx, axis=1)
    dhz = np.gradient(hgt, gz, axis=0)
    nrm = np.stack([-dhx, np.ones_like(hgt), -dhz], axis=-1).reshape(-1, 3)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    # triangles: quad (i,j) -> (a,b,c), (b,d,c)
    j, i = np.meshgrid(np.arange(nx), np.arange(ny))
    a = (i * (nx + 1) + j).ravel()
    b = a + 1
    c = a + (nx + 1)
    d = c + 1
    tris = np.stack([np.stack([a, b, c], 1), np.stack([b, d, c], 1)], 1).reshape(-1, 3)
    tilt = np.radians(6.0 + 4.0 * rng.uniform(1)[0])
    dist = sz / (np.tan(np.radians(30.0)) * overfill)
    eye = np.array([0.0, dist * np.cos(tilt), dist * np.sin(tilt)])
    mvp = _look_at_perspective(eye, [0.0, 0.0, 0.0], [0.0, 0.0, -1.0], 60.0, aspect,
                               0.25 * dist, 4.0 * dist)
    color = rng.uniform(3 * pos.shape[0]).reshape(-1, 3) if with_color else None
    return Scene(width, height, _f32(pos), _i32(tris),
                 color=None if color is None else _f32(color), normal=_f32(nrm),
                 mvp=_f32(mvp.ravel()), light_dir=listing1_light(),
                 shade_mode=shade_mode, name=f"heightfield{nx}x{ny}_{width}x{height}")


# --------------------------------------------------------------------------
# Power-law triangle sizes (1920x1080, 500k triangles, alpha = 2)
# --------------------------------------------------------------------------
def power_law_triangles(width=1920, height=1080, num_tris=500_000, seed=1237,
                        area_min=1.0, area_max_frac=0.25, shade_mode=SHADE_GBUFFER) -> Scene:
    """Triangles whose screen areas follow pdf(a) ~ a^-2 on [1 px^2, 1/4 screen],
    drawn by the inverse CDF, with aspect in [1,4], random orientation, a
    uniform centre, per-vertex depth on a small random slope, random unit
    normals facing the viewer and random albedo."""
    rng = SplitMix64(seed)
    T = int(num_tris)
    amax = area_max_frac * width * height
    u = rng.uniform(T)
    area = area_min / (1.0 - u * (1.0 - area_min / amax))
    aspect = 1.0 + 3.0 * rng.uniform(T)
    base = np.sqrt(2.0 * area / aspect)
    h = base * aspect
    apex = (rng.uniform(T) - 0.5) * base
    loc = np.stack([np.stack([-base / 2, np.zeros(T)], 1), np.stack([base / 2, np.zeros(T)], 1),
                    np.stack([apex, h], 1)], 1)                   # [T,3,2] pixels
    loc -= loc.mean(axis=1, keepdims=True)
    th = rng.uniform(T) * 2.0 * np.pi
    ct, st = np.cos(th)[:, None], np.sin(th)[:, None]
    rx = ct * loc[..., 0] - st * loc[..., 1]
    ry = st * loc[..., 0] + ct * loc[..., 1]
    cx = rng.uniform(T)[:, None] * width
    cy = rng.uniform(T)[:, None] * height
    px, py = cx + rx, cy + ry
    z0 = rng.uniform(T)[:, None] * 1.6 - 0.8
    slope = (rng.uniform(2 * T).reshape(T, 2) - 0.5) * (0.1 / max(width, height))
    z = np.clip(z0 + slope[:, :1] * rx + slope[:, 1:] * ry, -0.99, 0.99)
    x = px * (2.0 / width) - 1.0
    y = 1.0 - py * (2.0 / height)
    pos = np.stack([x, y, z, np.ones_like(x)], -1).reshape(3 * T, 4)
    v = rng.uniform(9 * T).reshape(3 * T, 3) * 2.0 - 1.0
    v[:, 2] = -np.abs(v[:, 2]) - 0.5
    nrm = v / np.linalg.norm(v, axis=1, keepdims=True)
    alb = rng.uniform(9 * T).reshape(3 * T, 3)
    return Scene(width, height, _f32(pos), _i32(np.arange(3 * T).reshape(T, 3)),
                 color=_f32(alb), normal=_f32(nrm), shade_mode=shade_mode,
                 name=f"powerlaw{T}_{width}x{height}")


def point_lights(width=1920, height=1080, n=64, seed=1241) -> np.ndarray:
    """n point lights as float32 [n,4] = (x, y, z, intensity): position uniform
    over the screen box times [-D/4, D/4] with D = max(width, height), and
    intensity uniform in [0, 1/16]."""
    rng = SplitMix64(seed)
    dz = float(max(width, height))
    p = rng.uniform(3 * n).reshape(n, 3)
    lights = np.stack([p[:, 0] * width, p[:, 1] * height, (p[:, 2] - 0.5) * 0.5 * dz,
                       rng.uniform(n) / 16.0], -1)
    return _f32(lights)


def gbuffer_inputs(width, height, seed=1242, empty_frac=0.2):
    """A synthetic G-buffer (key uint64, normal and albedo as float16 [H,W,4])
    for testing the light pass on its own: random depth and ID, a fraction of
    empty pixels (key = all ones), unit normals facing the viewer."""
    rng = SplitMix64(seed)
    n = width * height
    z = rng.integers(0, 1 << 24, n).astype(np.uint64)
    tid = rng.integers(0, 1 << 20, n).astype(np.uint64)
    key = (z << np.uint64(32)) | tid
    empty = rng.uniform(n) < empty_frac
    key[empty] = np.uint64(0xFFFFFFFFFFFFFFFF)
    v = rng.uniform(3 * n).reshape(n, 3) * 2.0 - 1.0
    v[:, 2] = -np.abs(v[:, 2]) - 0.3
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    nrm = np.zeros((n, 4), np.float16)
    nrm[:, :3] = v.astype(np.float16)
    alb = np.zeros((n, 4), np.float16)
    alb[:, :3] = rng.uniform(3 * n).reshape(n, 3).astype(np.float16)
    alb[:, 3] = 1.0
    nrm[empty] = 0
    alb[empty] = 0
    return (key.reshape(height, width), nrm.reshape(height, width, 4),
            alb.reshape(height, width, 4))


# --------------------------------------------------------------------------
# Tessellated sphere seen from 64 random cameras (512x512, ~100k triangles)
# --------------------------------------------------------------------------
def uv_sphere(slices=250, stacks=200):
    """Unit UV sphere: (stacks-1)*slices ring vertices plus two poles;
    2*slices cap triangles and 2*slices*(stacks-2) band triangles."""
    th = np.arange(1, stacks) * (np.pi / stacks)           # polar angle of each ring
    ph = np.arange(slices) * (2.0 * np.pi / slices)
    st, ct = np.sin(th)[:, None], np.cos(th)[:, None]
    ring = np.stack([st * np.cos(ph)[None, :], ct * np.ones_like(ph)[None, :],
                     st * np.sin(ph)[None, :]], -1).reshape(-1, 3)
    pts = np.concatenate([[[0.0, 1.0, 0.0]], ring, [[0.0, -1.0, 0.0]]], 0)
    top, bot = 0, pts.shape[0] - 1
    tri = []
    s = np.arange(slices)
    s1 = (s + 1) % slices
    tri.append(np.stack([np.full(slices, top), 1 + s1, 1 + s], 1))
    for r in range(stacks - 2):
        a = 1 + r * slices + s
        b = 1 + r * slices + s1
        c = 1 + (r + 1) * slices + s
        d = 1 + (r + 1) * slices + s1
        tri.append(np.stack([a, b, c], 1))
        tri.append(np.stack([b, d, c], 1))
    last = 1 + (stacks - 2) * slices
    tri.append(np.stack([last + s, last + s1, np.full(slices, bot)], 1))
    return pts, np.concatenate(tri, 0)


def sphere_views(num_views=64, width=512, height=512, slices=250, stacks=200, seed=1238):
    """The sphere with per-vertex colour and normals, a seeded unit light, and
    num_views cameras at distance 3 (FOV 60 degrees) looking at the centre.
    Returns (scene, mvps float32 [num_views,16])."""
    rng = SplitMix64(seed)
    pts, tris = uv_sphere(slices, stacks)
    V = pts.shape[0]
    pos = np.concatenate([pts, np.ones((V, 1))], 1)
    color = rng.uniform(3 * V).reshape(V, 3)
    L = rng.uniform(3) * 2.0 - 1.0
    L /= np.linalg.norm(L)
    mvps = []
    for _ in range(num_views):
        d = rng.uniform(3) * 2.0 - 1.0
        d /= max(np.linalg.norm(d), 1e-6)
        up = np.array([0.0, 1.0, 0.0]) if abs(d[1]) < 0.9 else np.array([1.0, 0.0, 0.0])
        mvps.append(_look_at_perspective(3.0 * d, [0.0, 0.0, 0.0], up, 60.0, width / height,
                                         1.0, 5.0).ravel())
    scene = Scene(width, height, _f32(pos), _i32(tris), color=_f32(color), normal=_f32(pts),
                  mvp=_f32(mvps[0]), light_dir=_f32(L), shade_mode=SHADE_LAMBERT,
                  name=f"sphere{tris.shape[0]}_{width}x{height}")
    return scene, _f32(np.stack(mvps))


def reyes_grids(width=1024, height=768, num_patches=256, seed=1243, micropoly_px=0.5, side_min=16.0,
                side_max=160.0, max_dice=128) -> Scene:
    """Micropolygon grids as a Reyes Dice stage would emit them (the input of
    the Sample stage, Sec. 7.1 of the Piko paper): seeded bicubic Bezier
    patches, each diced into an n x n grid of quads of about `micropoly_px`
    pixels a side (n = ceil(screen side / micropoly_px), capped at
    `max_dice`), every quad split into two triangles.  Patch screen sides
    are log-uniform in [side_min, side_max] pixels, centres uniform, control
    points on a random tilted plane with a seeded bulge; depth in NDC (w = 1).
    Per-vertex normals from the patch's partial derivatives and a per-patch
    albedo; Lambert with the light of Listing 1.  Split and Dice themselves
    are not part of this generator's output contract: only their result."""
    rng = SplitMix64(seed)
    P = int(num_patches)
    side = side_min * np.exp(rng.uniform(P) * np.log(side_max / side_min))
    cx = rng.uniform(P) * width
    cy = rng.uniform(P) * height
    z0 = rng.uniform(P) * 1.6 - 0.8
    tilt = (rng.uniform(2 * P).reshape(P, 2) - 0.5) * 0.6
    bulge = (rng.uniform(16 * P).reshape(P, 4, 4) - 0.5) * 0.5
    rot = rng.uniform(P) * 2.0 * np.pi
    alb = rng.uniform(3 * P).reshape(P, 3)
    # Bernstein basis of degree 3
    def bern(t):
        return np.stack([(1 - t) ** 3, 3 * t * (1 - t) ** 2, 3 * t ** 2 * (1 - t), t ** 3], -1)

    def dbern(t):
        return np.stack([-3 * (1 - t) ** 2, 3 * (1 - t) ** 2 - 6 * t * (1 - t), 6 * t * (1 - t) - 3 * t ** 2,
                         3 * t ** 2], -1)
    pos_l, tri_l, nrm_l, col_l = [], [], [], []
    base = 0
    for k in range(P):
        n = int(min(max_dice, max(1, np.ceil(side[k] / micropoly_px))))
        # control points: a square of side `side` in pixels, rotated, on a
        # tilted plane in depth with a bulge (depth units: NDC)
        g = np.linspace(-0.5, 0.5, 4)
        gu, gv = np.meshgrid(g, g, indexing="ij")
        ct, st = np.cos(rot[k]), np.sin(rot[k])
        px = cx[k] + side[k] * (ct * gu - st * gv)
        py = cy[k] + side[k] * (st * gu + ct * gv)
        pz = z0[k] + tilt[k, 0] * gu + tilt[k, 1] * gv + bulge[k] * 0.2
        C = np.stack([px * (2.0 / width) - 1.0, 1.0 - py * (2.0 / height), np.clip(pz, -0.95, 0.95)], -1)
        t = np.linspace(0.0, 1.0, n + 1)
        Bu, Bv, dBu, dBv = bern(t), bern(t), dbern(t), dbern(t)
        S = np.einsum("ia,jb,abc->ijc", Bu, Bv, C)
        Su = np.einsum("ia,jb,abc->ijc", dBu, Bv, C)
        Sv = np.einsum("ia,jb,abc->ijc", Bu, dBv, C)
        N = np.cross(Su, Sv)
        N /= np.maximum(np.linalg.norm(N, axis=-1, keepdims=True), 1e-12)
        N[..., 2] = -np.abs(N[..., 2])  # facing the viewer (-z)
        pos_l.append(np.concatenate([S.reshape(-1, 3), np.ones(((n + 1) ** 2, 1))], 1))
        nrm_l.append(N.reshape(-1, 3))
        col_l.append(np.tile(alb[k], ((n + 1) ** 2, 1)))
        j, i = np.meshgrid(np.arange(n), np.arange(n))
        a = (i * (n + 1) + j).ravel() + base
        b = a + 1
        c = a + (n + 1)
        d = c + 1
        tri_l.append(np.stack([np.stack([a, b, c], 1), np.stack([b, d, c], 1)], 1).reshape(-1, 3))
        base += (n + 1) ** 2
    return Scene(width, height, _f32(np.concatenate(pos_l)), _i32(np.concatenate(tri_l)),
                 color=_f32(np.concatenate(col_l)), normal=_f32(np.concatenate(nrm_l)),
                 light_dir=listing1_light(), shade_mode=SHADE_LAMBERT,
                 name=f"reyes{P}_{width}x{height}")


def target_image(width, height, seed=1240, views=1) -> np.ndarray:
    """A seeded target image float32 [views,H,W,4] in [0,1] for an L2 loss."""
    rng = SplitMix64(seed)
    return _f32(rng.uniform(views * height * width * 4).reshape(views, height, width, 4))


# --------------------------------------------------------------------------
# Many scenes with uneven sizes (256 scenes, 1k-200k triangles)
# --------------------------------------------------------------------------
def scene_batch(num_scenes=256, tmin=1_000, tmax=200_000, side_min=256, side_max=1024, seed=1239,
                shade_mode=SHADE_LAMBERT):
    """Scenes with triangle counts log-uniform in [tmin, tmax] and square
    sides uniform over the multiples of 64 in [side_min, side_max]; a seeded
    coin picks the random-triangle or the heightfield generator for each."""
    rng = SplitMix64(seed)
    scenes = []
    sides = np.arange(side_min, side_max + 1, 64)
    for k in range(num_scenes):
        T = int(round(np.exp(np.log(tmin) + rng.uniform(1)[0] * (np.log(tmax) - np.log(tmin)))))
        side = int(sides[rng.integers(0, len(sides), 1)[0]])
        sub_seed = int(rng.next_u64(1)[0] & np.uint64(0x7FFFFFFF))
        if rng.uniform(1)[0] < 0.5:
            # radius chosen so the expected covered area is a few screens' worth
            radius = float(np.clip(np.sqrt(3.0 * side * side / max(T, 1) / 0.2321), 2.0, 64.0))
            s = random_triangles(side, side, T, radius, seed=sub_seed, shade_mode=shade_mode,
                                 with_normals=True)
        else:
            q = max(1, int(round(np.sqrt(T / 2.0))))
            s = heightfield(side, side, q, max(1, T // (2 * q)), seed=sub_seed,
                            shade_mode=shade_mode, with_color=True)
        s.name = f"batch{k}_" + s.name
        scenes.append(s)
    return scenes


def config_scene(index: int, **kw):
    """The five workloads by number (1-based): 1 random 256x256 1k triangles,
    2 heightfield 1080p 1M, 3 power-law 1080p 500k (G-buffer), 4 sphere 64
    views, 5 batch of 256 scenes."""
    if index == 1:
        return random_triangles(**kw)
    if index == 2:
        return heightfield(**kw)
    if index == 3:
        return power_law_triangles(**kw)
    if index == 4:
        return sphere_views(**kw)
    if index == 5:
        return scene_batch(**kw)
    raise ValueError(index)
