"""Exact triangle-vs-bin overlap in AssignBin (PIKO_OPT_EXACT_BINS).

With the option on, a triangle spanning several bins gets an entry only in
the bins where none of its edges fails the fill-rule test at every pixel
centre of the bin inside its bounding box.  Keys and colours must stay
bit-exact / within 1e-5 of the oracle under every bin size and schedule;
the bin-entry count must fall for thin and large triangles and equal a
count of the same test done here on the oracle's snapped vertices; and a
triangle rendered alone must keep every bin in which it covers a pixel.
"""
import numpy as np
import pytest

import oracle
from binning_model import exact_bin_entries
from paper_1404_6293_gb300 import scenes as S

pytestmark = pytest.mark.gpu

RGB_TOL = 1e-5
EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


def _render(scene, bins, schedule, exact, extra=None):
    import torch
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene, Rasterizer
    r = Rasterizer(scene.width, scene.height, bins[0], bins[1], schedule)
    r.set_option(L.PIKO_OPT_EXACT_BINS, exact)
    r.set_option(L.PIKO_OPT_STATS, 1)
    for k, v in (extra or {}).items():
        r.set_option(k, v)
    ds = DeviceScene.from_host(scene)
    fb = r.forward(ds)
    torch.cuda.synchronize()
    code, _ = r.status()
    assert code == 0
    return fb.key_numpy(), (fb.rgba.cpu().numpy() if fb.rgba is not None else None), r.stats()["bin_entries"]


def _keys_equal(got, ref, what):
    bad = np.argwhere(got != ref)
    assert bad.size == 0, f"{what}: {len(bad)} keys differ, first at {tuple(bad[0][::-1])}"


def _model_entries(scene, bw, bh):
    return exact_bin_entries(scene, bw, bh)


def _thin_scene(W, H, T, seed):
    """Long thin triangles at every angle across the frame, and a few large ones."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.1, 0.9, (T, 2)) * [W, H]
    ang = rng.uniform(0, np.pi, T)
    length = rng.uniform(0.3, 1.2, T) * max(W, H)
    width = np.where(rng.random(T) < 0.8, rng.uniform(0.5, 3.0, T), rng.uniform(20, 80, T))
    d = np.stack([np.cos(ang), np.sin(ang)], 1)
    n = np.stack([-d[:, 1], d[:, 0]], 1)
    p0 = c - d * length[:, None] / 2
    p1 = c + d * length[:, None] / 2
    p2 = c + n * width[:, None]
    px = np.stack([p0[:, 0], p1[:, 0], p2[:, 0]], 1)
    py = np.stack([p0[:, 1], p1[:, 1], p2[:, 1]], 1)
    z = rng.integers(0, 1 << 24, (T, 3)) * (2.0 / 16777215.0) - 1.0
    pos = np.stack([px / W * 2 - 1, 1 - py / H * 2, z, np.ones_like(z)], -1).reshape(3 * T, 4)
    return S.Scene(W, H, pos.astype(np.float32), np.arange(3 * T, dtype=np.int32).reshape(T, 3),
                   color=rng.random((3 * T, 3)).astype(np.float32), name=f"thin{T}_{W}x{H}")


SCENES = {
    "thin": lambda: _thin_scene(203, 141, 120, seed=5),
    "power_law": lambda: S.power_law_triangles(256, 160, 1500, seed=44, shade_mode=S.SHADE_GOURAUD),
    "random_large": lambda: S.random_triangles(190, 130, 200, 70.0, seed=81),
}


@pytest.mark.parametrize("name", sorted(SCENES))
@pytest.mark.parametrize("bins", [(8, 8), (16, 16), (32, 32), (64, 16)])
def test_exact_bins_match_oracle_with_fewer_entries(name, bins):
    s = SCENES[name]()
    ref, _ = oracle.raster_bbox(s, threads=4)
    rgba_ref = oracle.shade(s, ref)
    want = _model_entries(s, *bins)
    for sched in ("static", "dynamic", "hardware"):
        key0, _, e0 = _render(s, bins, sched, 0)
        key1, rgba1, e1 = _render(s, bins, sched, 1)
        _keys_equal(key0, ref, f"{name} {bins} {sched} bounding-box bins")
        _keys_equal(key1, ref, f"{name} {bins} {sched} exact bins")
        assert np.abs(rgba1 - rgba_ref).max() <= RGB_TOL
        assert e1 == want, (name, bins, sched, e1, want)
        assert e1 <= e0
    if name == "thin" and bins[0] <= 16:
        assert e1 < 0.8 * e0, (e1, e0)  # thin diagonals leave most of their boxes' bins


def test_each_triangle_alone_keeps_every_bin_it_covers():
    """One thin triangle per frame: nothing occludes it, so every pixel it
    covers is in the key buffer, and each bin holding such a pixel must have
    kept its entry (else the keys would differ)."""
    full = _thin_scene(150, 100, 24, seed=9)
    for t in range(full.num_triangles):
        tri = full.tris[t]
        s = S.Scene(full.width, full.height, full.pos[tri], np.arange(3, dtype=np.int32).reshape(1, 3),
                    color=full.color[tri], name=f"thin_alone_{t}")
        ref, _ = oracle.raster_bbox(s)
        covered = np.argwhere(ref != EMPTY)
        for bins in ((8, 8), (16, 16)):
            key, _, e = _render(s, bins, "dynamic", 1)
            _keys_equal(key, ref, f"triangle {t} alone, bins {bins}")
            bins_hit = {(int(y) // bins[1], int(x) // bins[0]) for y, x in covered}
            assert len(bins_hit) <= e == _model_entries(s, *bins)


def test_exact_bins_with_near_far_clipping():
    from paper_1404_6293_gb300 import _lib as L
    rng = np.random.default_rng(31)
    T, W, H = 300, 150, 104
    xy = rng.uniform(-1.3, 1.3, (3 * T, 2))
    w = rng.uniform(0.2, 2.0, 3 * T)
    w[rng.random(3 * T) < 0.1] *= -1.0
    z = rng.uniform(-1.6, 1.6, 3 * T) * np.abs(w)
    pos = np.stack([xy[:, 0] * w, xy[:, 1] * w, z, w], 1).astype(np.float32)
    s = S.Scene(W, H, pos, np.arange(3 * T, dtype=np.int32).reshape(T, 3),
                color=rng.random((3 * T, 3)).astype(np.float32), name="clip_exact")
    oracle.set_clipping(True)
    try:
        ref, _ = oracle.raster_bbox(s)
    finally:
        oracle.set_clipping(False)
    for sched in ("static", "dynamic"):
        key0, _, e0 = _render(s, (16, 16), sched, 0, {L.PIKO_OPT_CLIP: 1})
        key1, _, e1 = _render(s, (16, 16), sched, 1, {L.PIKO_OPT_CLIP: 1})
        _keys_equal(key0, ref, f"clipping {sched}")
        _keys_equal(key1, ref, f"clipping + exact bins {sched}")
        assert e1 <= e0


@pytest.mark.parametrize("exact", [0, 1])
def test_heavy_triangles_without_the_list(exact):
    """Triangles spanning 256 bins or more are listed for the scatter pass;
    with the list treated as full (test hook bit 2) their entries are
    written by their own warps instead.  Same keys and entry counts either
    way, and equal to the oracle."""
    from paper_1404_6293_gb300 import _lib as L
    s = S.random_triangles(400, 300, 150, 160.0, seed=17)
    ref, _ = oracle.raster_bbox(s, threads=4)
    out = []
    for hook in (0, 4):
        for sched in ("static", "hardware"):
            key, _, e = _render(s, (8, 8), sched, exact, {L.PIKO_OPT_TEST_WITHHOLD: hook})
            _keys_equal(key, ref, f"heavy list hook={hook} {sched} exact={exact}")
            out.append(e)
    assert len(set(out)) == 1
    if exact:
        assert out[0] == _model_entries(s, 8, 8)
