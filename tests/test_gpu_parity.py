"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Depth/ID keys must match bit for bit; shaded colour within 1e-5 absolute
(the GPU shades in float32, the oracle in float64); binary16 G-buffer
values within one binary16 step (both sides round a value that differs only
by float32-vs-float64 interpolation); gradients within 1e-4 relative on
components above 1e-3 of the largest, 1e-4 of the largest below that.
"""
import numpy as np
import pytest

import oracle
from paper_1404_6293_gb300 import scenes as S

pytestmark = pytest.mark.gpu

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)
RGB_TOL = 1e-5


def _torch():
    import torch
    return torch


def rasterize(scene, bin_w=16, bin_h=16, schedule="static", options=None, mvp=None):
    torch = _torch()
    from paper_1404_6293_gb300.raster import DeviceScene, Rasterizer
    r = Rasterizer(scene.width, scene.height, bin_w, bin_h, schedule)
    for k, v in (options or {}).items():
        r.set_option(k, v)
    ds = DeviceScene.from_host(scene, mvp=mvp)
    fb = r.forward(ds)
    torch.cuda.synchronize()
    code, need = r.status()
    out = {"key": fb.key_numpy(), "status": code, "needed": need, "r": r, "ds": ds, "fb": fb}
    if fb.rgba is not None:
        out["rgba"] = fb.rgba.cpu().numpy()
    if fb.gbuf_normal is not None:
        out["gn"] = fb.gbuf_normal.cpu().numpy()
        out["ga"] = fb.gbuf_albedo.cpu().numpy()
    return out


def assert_keys_equal(gpu, ref, what=""):
    if not np.array_equal(gpu, ref):
        bad = np.argwhere(gpu != ref)
        y, x = bad[0]
        raise AssertionError(f"{what}: {len(bad)} key mismatches, first at (x={x}, y={y}): "
                             f"gpu {int(gpu[y, x]):#x} oracle {int(ref[y, x]):#x}")


# Both sides round to binary16 a value that differs only by the float32
# (GPU) versus float64 (oracle) interpolation, at most HALF_INTERP_ERR apart
# for the O(1) attributes here; rounding two values that far apart gives
# codes at most one binary16 step plus that distance apart.  Near zero,
# where the step is a subnormal 2^-24, the distance term dominates.
HALF_INTERP_ERR = 1e-6


def assert_half_close(gpu_h, ref_u16):
    g = gpu_h.astype(np.float64)
    r = ref_u16.view(np.float16).astype(np.float64)
    step = np.spacing(np.maximum(np.abs(g), np.abs(r)).astype(np.float16)).astype(np.float64)
    lim = step + HALF_INTERP_ERR
    assert np.all(np.abs(g - r) <= lim), np.max(np.abs(g - r) / lim)


# --------------------------------------------------------------- configs
def test_random_triangles_256_parity():
    s = S.random_triangles()
    out = rasterize(s, 16, 16, "static")
    assert out["status"] == 0
    ref, st = oracle.raster_brute(s)
    assert st == 0
    assert_keys_equal(out["key"], ref, "random 256x256")
    rgba = oracle.shade(s, ref)
    assert np.abs(out["rgba"] - rgba).max() <= RGB_TOL


SHAPES = [(1, 1), (7, 5), (37, 53), (200, 120), (257, 65), (64, 64)]


@pytest.mark.parametrize("W,H", SHAPES)
@pytest.mark.parametrize("bins", [(8, 8), (16, 16), (32, 32), (64, 64), (8, 32), (64, 16)])
def test_all_bins_and_schedules_match_oracle(W, H, bins):
    rng = np.random.default_rng(W * 1000 + H)
    T = int(rng.integers(50, 400))
    radius = float(rng.choice([3.0, 12.0, 60.0, 300.0]))
    s = S.random_triangles(W, H, T, radius, seed=int(rng.integers(1 << 30)))
    ref, _ = oracle.raster_bbox(s, threads=4)
    rgba_ref = oracle.shade(s, ref)
    for sched in ("static", "dynamic", "hardware"):
        out = rasterize(s, bins[0], bins[1], sched)
        assert out["status"] == 0
        assert_keys_equal(out["key"], ref, f"{W}x{H} bins {bins} {sched}")
        assert np.abs(out["rgba"] - rgba_ref).max() <= RGB_TOL


@pytest.mark.parametrize("small_px", [0, 1, 32, 4096])
@pytest.mark.parametrize("threads", [64, 128, 256, 512])
def test_thread_and_warp_raster_paths_agree(small_px, threads):
    from paper_1404_6293_gb300 import _lib as L
    s = S.random_triangles(160, 96, 300, 25.0, seed=77)
    ref, _ = oracle.raster_bbox(s)
    out = rasterize(s, 32, 16, "dynamic", {L.PIKO_OPT_SMALL_TRI_PIXELS: small_px, L.PIKO_OPT_THREADS_PER_TILE: threads})
    assert_keys_equal(out["key"], ref, f"small_px={small_px} threads={threads}")


@pytest.mark.parametrize("W,H,bins", [(256, 256, 16), (640, 480, 16), (1024, 512, 16), (1024, 528, 16), (200, 120, 8)])
def test_count_pass_scan_matches_scan_kernel(W, H, bins):
    """A frame of at most 2,048 bins is scanned by the count pass's last CTA;
    with stage events on, the forward keeps the count and scan launches
    apart.  Both give the same keys, colours and bin-entry total as the
    oracle, frame after frame (the fused pass resets its CTA counter)."""
    torch = _torch()
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene, Framebuffer, Rasterizer
    s = S.random_triangles(W, H, 2000, 20.0, seed=W + H)
    ref, _ = oracle.raster_bbox(s, threads=4)
    rgba_ref = oracle.shade(s, ref)
    r = Rasterizer(W, H, bins, bins, "hardware")
    r.set_option(L.PIKO_OPT_STATS, 1)
    ds = DeviceScene.from_host(s)
    fb = Framebuffer.allocate(W, H, s.shade_mode)
    entries = []
    for step in range(4):
        if step % 2:
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(L.PIKO_NUM_STAGE_EVENTS)]
            for e in ev:
                e.record()  # creates the CUDA events
            r.set_stage_events(ev)
        fb.key.fill_(0)
        r.forward(ds, fb)
        torch.cuda.synchronize()
        assert r.status()[0] == 0
        assert_keys_equal(fb.key_numpy(), ref, f"{W}x{H} bins {bins} step {step}")
        assert np.abs(fb.rgba.cpu().numpy() - rgba_ref).max() <= RGB_TOL
        entries.append(r.stats()["bin_entries"])
    assert len(set(entries)) == 1


def _dense_small_boxes(W, H, T, seed):
    """Right triangles with legs 4.9 x 5.9 px (boxes of at most 5 x 6 pixel
    centres) at random places and orientations, about seven deep."""
    rng = np.random.default_rng(seed)
    cx = rng.uniform(0, W - 5, T)
    cy = rng.uniform(0, H - 6, T)
    fx = rng.random(T) < 0.5
    fy = rng.random(T) < 0.5
    ax = np.where(fx, cx + 4.9, cx)
    bx = np.where(fx, cx, cx + 4.9)
    ay = np.where(fy, cy + 5.9, cy)
    cy2 = np.where(fy, cy, cy + 5.9)
    px = np.stack([ax, bx, ax], 1)
    py = np.stack([ay, ay, cy2], 1)
    z = rng.integers(0, 1 << 24, (T, 3)) * (2.0 / 16777215.0) - 1.0
    pos = np.stack([px / W * 2 - 1, 1 - py / H * 2, z, np.ones_like(z)], -1).reshape(3 * T, 4)
    color = rng.random((3 * T, 3))
    return S.Scene(W, H, pos.astype(np.float32), np.arange(3 * T, dtype=np.int32).reshape(T, 3),
                   color=color.astype(np.float32), name=f"dense{T}_{W}x{H}")


@pytest.mark.parametrize("bins", [(8, 8), (16, 16), (64, 64), (32, 8)])
def test_dense_small_boxes_many_fragments_per_warp(bins):
    """Small boxes seven deep: a warp's boxes hold hundreds of covered
    samples, so the warp hands them out over several rounds of its fragment
    list.  Keys bit-exact and colour within 1e-5 under each raster path
    (boxes by the warp's compacted fragments, by one thread each, by whole
    warps), with the same fragment count."""
    from paper_1404_6293_gb300 import _lib as L
    s = _dense_small_boxes(99, 70, 3000, seed=4242 + bins[0])
    ref, _ = oracle.raster_bbox(s)
    rgba_ref = oracle.shade(s, ref)
    counts = []
    for small_px in (32, 4096, 0):
        out = rasterize(s, bins[0], bins[1], "dynamic",
                        {L.PIKO_OPT_SMALL_TRI_PIXELS: small_px, L.PIKO_OPT_STATS: 1})
        assert out["status"] == 0
        assert_keys_equal(out["key"], ref, f"bins {bins} small_px={small_px}")
        assert np.abs(out["rgba"] - rgba_ref).max() <= RGB_TOL
        counts.append(out["r"].stats()["fragments"])
    assert counts[0] == counts[1] == counts[2] > 0


def test_lambert_heightfield_small():
    s = S.heightfield(320, 180, 80, 40, seed=5)
    ref, _ = oracle.raster_bbox(s, threads=4)
    rgba = oracle.shade(s, ref)
    for bins in ((8, 8), (16, 16), (64, 64)):
        out = rasterize(s, *bins)
        assert_keys_equal(out["key"], ref, f"heightfield bins {bins}")
        assert np.abs(out["rgba"] - rgba).max() <= RGB_TOL


def test_lambert_with_colours_and_unclamped():
    from paper_1404_6293_gb300 import _lib as L
    s = S.random_triangles(128, 128, 200, 20.0, seed=8, shade_mode=S.SHADE_LAMBERT, with_normals=True)
    s.light_dir = np.array([0.2, -0.5, -0.84], np.float32)
    ref, _ = oracle.raster_brute(s)
    for unclamped in (0, 1):
        out = rasterize(s, 16, 16, "dynamic", {L.PIKO_OPT_UNCLAMPED: unclamped})
        assert_keys_equal(out["key"], ref)
        rgba = oracle.shade(s, ref, unclamped=bool(unclamped))
        assert np.abs(out["rgba"] - rgba).max() <= RGB_TOL


def test_heightfield_1080p_full_frame():
    s = S.heightfield()
    ref, _ = oracle.raster_bbox(s, threads=8)
    rgba = oracle.shade(s, ref)
    for bins in ((8, 8), (16, 16), (32, 32), (64, 64)):
        out = rasterize(s, *bins)
        assert out["status"] == 0
        assert_keys_equal(out["key"], ref, f"heightfield 1080p bins {bins}")
        assert np.abs(out["rgba"] - rgba).max() <= RGB_TOL


def test_gbuffer_power_law_small():
    s = S.power_law_triangles(480, 270, 20_000, seed=9)
    ref, _ = oracle.raster_bbox(s, threads=4)
    gn, ga = oracle.shade(s, ref)
    for sched in ("static", "dynamic"):
        out = rasterize(s, 16, 16, sched)
        assert_keys_equal(out["key"], ref, f"power law {sched}")
        assert_half_close(out["gn"], gn)
        assert_half_close(out["ga"], ga)


def test_power_law_1080p_full_frame_keys():
    s = S.power_law_triangles()
    ref, _ = oracle.raster_bbox(s, threads=8)
    out = rasterize(s, 16, 16, "dynamic")
    assert_keys_equal(out["key"], ref, "power law 1080p")


def test_deferred_light_pass_on_synthetic_gbuffer():
    torch = _torch()
    from paper_1404_6293_gb300.raster import Framebuffer, Rasterizer
    W, H = 333, 187
    key, gn, ga = S.gbuffer_inputs(W, H)
    lights = S.point_lights(W, H, 64)
    ref = oracle.light_pass(key, gn.view(np.uint16), ga.view(np.uint16), lights)
    r = Rasterizer(W, H, 16, 16)
    fb = Framebuffer(torch.from_numpy(key.view(np.int64)).cuda(), None, torch.from_numpy(gn).cuda(),
                     torch.from_numpy(ga).cuda())
    for n in (1, 7, 64):
        lt = lights[:n]
        ref = oracle.light_pass(key, gn.view(np.uint16), ga.view(np.uint16), lt)
        out = r.deferred_light(fb, torch.from_numpy(lt).cuda()).cpu().numpy()
        assert np.abs(out - ref).max() <= RGB_TOL


def test_deferred_end_to_end_where_gbuffer_agrees():
    torch = _torch()
    s = S.power_law_triangles(480, 270, 20_000, seed=10)
    lights = S.point_lights(480, 270, 64)
    ref_key, _ = oracle.raster_bbox(s)
    gn, ga = oracle.shade(s, ref_key)
    ref = oracle.light_pass(ref_key, gn, ga, lights)
    out = rasterize(s, 16, 16, "dynamic")
    assert_keys_equal(out["key"], ref_key, "deferred G-buffer keys")
    rgba = out["r"].deferred_light(out["fb"], torch.from_numpy(lights).cuda()).cpu().numpy()
    # the G-buffer contract: every binary16 word within one step of the oracle's
    assert_half_close(out["gn"], gn)
    assert_half_close(out["ga"], ga)
    same = np.all(out["gn"].view(np.uint16) == gn, axis=-1) & np.all(out["ga"].view(np.uint16) == ga, axis=-1)
    assert same.mean() > 0.99
    assert np.abs(rgba[same] - ref[same]).max() <= RGB_TOL
    # Where a word differs, the light pass sees albedo a + da and normal
    # n + dn with |da_c|, |dn_c| <= h = 2^-11 + HALF_INTERP_ERR (one binary16
    # step below 1, plus the interpolation difference; every albedo and
    # normal component here is below 1).  The light sum
    # S = sum_l I_l max(0, n . d_l) / (1 + |d_l|^2 / r^2) then moves by at
    # most sum_l I_l |dn| <= sqrt(3) h sum_l I_l, so
    # |d rgb_c| <= h S + a_c sqrt(3) h sum_l I_l <= (1 + sqrt(3)) h sum_l I_l.
    h = 2.0 ** -11 + HALF_INTERP_ERR
    assert max(np.abs(gn.view(np.float16)).max(), np.abs(ga[..., :3].view(np.float16)).max()) < 1.0
    bound = (1.0 + np.sqrt(3.0)) * h * float(lights[:, 3].astype(np.float64).sum()) + RGB_TOL
    assert np.abs(rgba - ref).max() <= bound


# --------------------------------------------------------------- edge cases
def test_empty_scene_and_no_vertices():
    for V, T in ((0, 0), (30, 0)):
        s = S.Scene(40, 30, np.zeros((V, 4), np.float32), np.zeros((T, 3), np.int32),
                    color=np.zeros((V, 3), np.float32))
        out = rasterize(s, 8, 8)
        assert out["status"] == 0
        assert (out["key"] == EMPTY).all()
        assert (out["rgba"] == 0).all()


def test_culled_degenerate_and_huge_triangles():
    W = H = 256
    pos = []
    # huge triangle (A > 2^38: 128-bit depth path), vertices near the guard band
    pos += [[-200.0, -200.0, -0.5, 1], [200.0, -200.0, 0.7, 1], [0.0, 230.0, 0.1, 1]]
    # vertex behind the camera (w < 0) and one with z outside [-1, 1]
    pos += [[0, 0, 0, -1], [0.5, 0, 0, 1], [0, 0.5, 0, 1]]
    pos += [[0, 0, 1.5, 1], [0.5, 0, 0, 1], [0, 0.5, 0, 1]]
    # collinear (A = 0)
    pos += [[-0.5, -0.5, 0, 1], [0.0, 0.0, 0, 1], [0.5, 0.5, 0, 1]]
    # ordinary triangle in front of the huge one, and one behind it
    pos += [[-0.3, -0.3, -0.9, 1], [0.4, -0.2, -0.9, 1], [0.0, 0.5, -0.9, 1]]
    pos += [[-0.6, -0.1, 0.99, 1], [0.2, -0.7, 0.99, 1], [0.3, 0.6, 0.99, 1]]
    pos = np.array(pos, np.float32)
    n = pos.shape[0]
    rng = np.random.default_rng(0)
    s = S.Scene(W, H, pos, np.arange(n).reshape(-1, 3).astype(np.int32), color=rng.random((n, 3)).astype(np.float32))
    ref, _ = oracle.raster_brute(s)
    assert (ref != EMPTY).all()  # the huge triangle covers the screen
    for bins in ((8, 8), (64, 64)):
        for sched in ("static", "dynamic", "hardware"):
            out = rasterize(s, *bins, sched)
            assert_keys_equal(out["key"], ref, f"huge/culled {bins} {sched}")
            assert np.abs(out["rgba"] - oracle.shade(s, ref)).max() <= RGB_TOL


def test_bad_index_is_reported_and_culled():
    from paper_1404_6293_gb300 import _lib as L
    s = S.random_triangles(64, 64, 50, 10.0, seed=2)
    s.tris = s.tris.copy()
    s.tris[7] = [0, 1, 1 << 20]
    s.tris[9] = [-5, 2, 3]
    ref, st = oracle.raster_brute(s)
    assert st == oracle.BAD_INDEX
    out = rasterize(s, 16, 16)
    assert out["status"] == L.PIKO_ERR_BAD_INDEX
    assert_keys_equal(out["key"], ref, "bad index")


def test_overflow_is_reported_then_grows():
    torch = _torch()
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene, Rasterizer
    s = S.random_triangles(256, 256, 2000, 40.0, seed=4)
    ref, _ = oracle.raster_bbox(s)
    r = Rasterizer(256, 256, 8, 8, "dynamic")
    r.set_option(L.PIKO_OPT_CHECK_CAPACITY, 0)
    r.reserve(s.num_vertices, s.num_triangles, 100)
    ds = DeviceScene.from_host(s)
    r.forward(ds)
    code, need = r.status()
    assert code == L.PIKO_ERR_OVERFLOW and need > 100
    r.reserve(s.num_vertices, s.num_triangles, need)
    fb = r.forward(ds)
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    assert_keys_equal(fb.key_numpy(), ref, "after reserve")
    # with the capacity check on, a too-small reservation grows by itself
    r2 = Rasterizer(256, 256, 8, 8, "static")
    r2.reserve(s.num_vertices, s.num_triangles, 10)
    fb2 = r2.forward(ds)
    torch.cuda.synchronize()
    assert r2.status()[0] == 0
    assert_keys_equal(fb2.key_numpy(), ref, "auto grow")


def test_invalid_arguments_rejected_on_host():
    torch = _torch()
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene, PikoError, Rasterizer
    lib = L.load()
    assert not lib.piko_raster_create(0, 10, 16, 16, 0)
    assert not lib.piko_raster_create(10, 10, 12, 16, 0)
    assert not lib.piko_raster_create(40000, 10, 16, 16, 0)
    assert not lib.piko_raster_create(10, 10, 16, 16, 7)
    r = Rasterizer(64, 64)
    s = S.random_triangles(32, 32, 5, 5.0)
    with pytest.raises(PikoError):
        r.forward(DeviceScene.from_host(s))  # size mismatch
    with pytest.raises(PikoError):
        r.set_option(L.PIKO_OPT_THREADS_PER_TILE, 100)
    s = S.random_triangles(64, 64, 5, 5.0)
    ds = DeviceScene.from_host(s)
    ds.color = None
    with pytest.raises(PikoError):
        r.forward(ds)  # Gouraud without colours


@pytest.mark.parametrize("W,H", [(32767, 3), (5, 32767)])
def test_largest_framebuffer_sides(W, H):
    """The widest and tallest framebuffers the 16.8 guard band allows
    (32767 pixels: snapped coordinates just below 2^23), with triangles that
    reach past the far edges; 32768 is rejected."""
    from paper_1404_6293_gb300 import _lib as L
    lib = L.load()
    assert not lib.piko_raster_create(W + 1 if W == 32767 else W, H + 1 if H == 32767 else H, 16, 16, 0)
    s = S.random_triangles(W, H, 400, 12.0, seed=90 + W)
    ref, _ = oracle.raster_bbox(s)
    assert (ref != EMPTY).any()
    for bins, sched in (((8, 8), "static"), ((64, 64), "dynamic"), ((16, 16), "hardware")):
        out = rasterize(s, *bins, sched)
        assert out["status"] == 0
        assert_keys_equal(out["key"], ref, f"{W}x{H} bins {bins} {sched}")


def test_bin_size_and_schedule_never_change_output():
    s = S.random_triangles(300, 200, 3000, 15.0, seed=12)
    keys = []
    for bins in ((8, 8), (16, 16), (32, 32), (64, 64), (16, 64)):
        for sched in ("static", "dynamic", "hardware"):
            keys.append(rasterize(s, *bins, sched)["key"])
    for k in keys[1:]:
        assert np.array_equal(k, keys[0])


# --------------------------------------------------------------- backward
def _grad_check(g_gpu, g_ref):
    g_gpu = np.asarray(g_gpu, np.float64)
    scale = np.abs(g_ref).max()
    big = np.abs(g_ref) > 1e-3 * scale
    rel = np.abs(g_gpu - g_ref)[big] / np.abs(g_ref)[big]
    assert rel.max() <= 1e-4, rel.max()
    assert np.abs(g_gpu - g_ref)[~big].max(initial=0) <= 1e-4 * scale


@pytest.mark.parametrize("mode", [S.SHADE_GOURAUD, S.SHADE_LAMBERT])
def test_backward_matches_oracle_gradients(mode):
    torch = _torch()
    s = S.random_triangles(128, 96, 400, 14.0, seed=31, shade_mode=mode, with_normals=True)
    s.light_dir = np.array([0.3, -0.4, -0.866], np.float32)
    out = rasterize(s, 16, 16, "dynamic")
    ref_key, _ = oracle.raster_brute(s)
    assert_keys_equal(out["key"], ref_key)
    tgt = S.target_image(128, 96, seed=2)[0]
    rgba_ref = oracle.shade(s, ref_key)
    g = np.zeros((96, 128, 4))
    g[..., :3] = 2.0 * (rgba_ref[..., :3] - tgt[..., :3])
    dc, dn, dl = oracle.backward(s, ref_key, g)
    V = s.num_vertices
    gd = torch.from_numpy(g.astype(np.float32)).cuda()
    dcg = torch.zeros((V, 3), device="cuda")
    dng = torch.zeros((V, 3), device="cuda")
    dlg = torch.zeros(3, device="cuda")
    out["r"].backward(out["ds"], out["fb"], gd, dcg, dng, dlg)
    torch.cuda.synchronize()
    _grad_check(dcg.cpu().numpy(), dc)
    if mode == S.SHADE_LAMBERT:
        _grad_check(dng.cpu().numpy(), dn)
        _grad_check(dlg.cpu().numpy(), dl)


# Two scene shapes select the two backward forms: few large triangles (per
# 16x16 tile, a shared table of distinct triangles) and more than one triangle
# per four pixels (per pixel).  Both against the oracle's gradients.
@pytest.mark.parametrize("shape", ["large", "tiny"])
def test_backward_tile_and_pixel_forms_match_oracle(shape):
    torch = _torch()
    if shape == "large":
        s = S.random_triangles(160, 112, 150, 40.0, seed=77, shade_mode=S.SHADE_LAMBERT, with_normals=True)
        assert 4 * s.num_triangles <= s.width * s.height
    else:
        s = S.heightfield(96, 80, 60, 40, seed=78, shade_mode=S.SHADE_LAMBERT, with_color=True)
        assert 4 * s.num_triangles > s.width * s.height
    out = rasterize(s, 16, 16, "static")
    ref_key, _ = oracle.raster_brute(s)
    assert_keys_equal(out["key"], ref_key)
    tgt = S.target_image(s.width, s.height, seed=5)[0]
    g = np.zeros((s.height, s.width, 4))
    g[..., :3] = 2.0 * (oracle.shade(s, ref_key)[..., :3] - tgt[..., :3])
    dc, dn, dl = oracle.backward(s, ref_key, g)
    V = s.num_vertices
    dcg = torch.zeros((V, 3), device="cuda")
    dng = torch.zeros((V, 3), device="cuda")
    dlg = torch.zeros(3, device="cuda")
    out["r"].backward(out["ds"], out["fb"], torch.from_numpy(g.astype(np.float32)).cuda(), dcg, dng, dlg)
    torch.cuda.synchronize()
    if s.color is not None:
        _grad_check(dcg.cpu().numpy(), dc)
    _grad_check(dng.cpu().numpy(), dn)
    _grad_check(dlg.cpu().numpy(), dl)


def test_autograd_render_gradients_match_oracle():
    torch = _torch()
    from paper_1404_6293_gb300.autograd import render
    from paper_1404_6293_gb300.raster import DeviceScene, Rasterizer
    s = S.random_triangles(96, 80, 300, 12.0, seed=41, shade_mode=S.SHADE_LAMBERT, with_normals=True)
    s.light_dir = np.array([0.2, -0.3, -0.93], np.float32)
    r = Rasterizer(s.width, s.height, 16, 16, "dynamic")
    ds = DeviceScene.from_host(s)
    color = ds.color.clone().requires_grad_(True)
    normal = ds.normal.clone().requires_grad_(True)
    light = ds.light_dir.clone().requires_grad_(True)
    rgba, key = render(r, ds, color, normal, light)
    tgt = torch.from_numpy(S.target_image(96, 80, seed=5)[0]).cuda()
    loss = ((rgba[..., :3] - tgt[..., :3]) ** 2).sum()
    loss.backward()
    ref_key, _ = oracle.raster_brute(s)
    assert_keys_equal(key.cpu().numpy().view(np.uint64), ref_key)
    rgba_ref = oracle.shade(s, ref_key)
    g = np.zeros((80, 96, 4))
    g[..., :3] = 2.0 * (rgba_ref[..., :3] - tgt.cpu().numpy()[..., :3])
    dc, dn, dl = oracle.backward(s, ref_key, g)
    _grad_check(color.grad.cpu().numpy(), dc)
    _grad_check(normal.grad.cpu().numpy(), dn)
    _grad_check(light.grad.cpu().numpy(), dl)
    # the loss itself agrees with the float64 oracle
    ref_loss = oracle.loss(s, ref_key, tgt.cpu().numpy())
    assert abs(loss.item() - ref_loss) <= 1e-4 * max(1.0, ref_loss)


def test_sphere_views_backward_accumulates_over_views():
    torch = _torch()
    from paper_1404_6293_gb300.autograd import render
    from paper_1404_6293_gb300.raster import DeviceScene, Rasterizer
    sph, mvps = S.sphere_views(num_views=3, width=128, height=128, slices=60, stacks=40)
    r = Rasterizer(128, 128, 16, 16, "dynamic")
    ds = DeviceScene.from_host(sph)
    color = ds.color.clone().requires_grad_(True)
    normal = ds.normal.clone().requires_grad_(True)
    light = ds.light_dir.clone().requires_grad_(True)
    tgt = torch.from_numpy(S.target_image(128, 128, seed=9, views=3)).cuda()
    total = 0.0
    dc_ref = np.zeros((sph.num_vertices, 3))
    dn_ref = np.zeros((sph.num_vertices, 3))
    dl_ref = np.zeros(3)
    for v in range(3):
        ds.mvp = torch.from_numpy(mvps[v]).cuda()
        rgba, key = render(r, ds, color, normal, light)
        loss = ((rgba[..., :3] - tgt[v, ..., :3]) ** 2).sum()
        loss.backward()
        total += loss.item()
        sv = S.Scene(128, 128, sph.pos, sph.tris, color=sph.color, normal=sph.normal, mvp=mvps[v],
                     light_dir=sph.light_dir, shade_mode=sph.shade_mode)
        ref_key, _ = oracle.raster_bbox(sv)
        assert_keys_equal(key.cpu().numpy().view(np.uint64), ref_key, f"view {v}")
        rgba_ref = oracle.shade(sv, ref_key)
        g = np.zeros((128, 128, 4))
        g[..., :3] = 2.0 * (rgba_ref[..., :3] - tgt[v].cpu().numpy()[..., :3])
        oracle.backward(sv, ref_key, g, out=(dc_ref, dn_ref, dl_ref))
    _grad_check(color.grad.cpu().numpy(), dc_ref)
    _grad_check(normal.grad.cpu().numpy(), dn_ref)
    _grad_check(light.grad.cpu().numpy(), dl_ref)


def test_sphere_views_as_one_batch_share_gradients():
    """The multi-view form the sphere workload is measured in: all views in
    one forward_batch / backward_batch, every view accumulating into the same
    mesh gradients; against the oracle summed over the views."""
    torch = _torch()
    import dataclasses
    from paper_1404_6293_gb300.raster import DeviceScene, Framebuffer, Rasterizer
    nv, W = 6, 128
    sph, mvps = S.sphere_views(num_views=nv, width=W, height=W, slices=60, stacks=40)
    ds = DeviceScene.from_host(sph)
    mv = torch.from_numpy(mvps).cuda()
    views = [dataclasses.replace(ds, mvp=mv[v]) for v in range(nv)]
    r = Rasterizer(64, 64)
    fbs = r.forward_batch(views, None, [(16, 16)] * nv, ["dynamic", "static"] * (nv // 2))
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    tgt = S.target_image(W, W, seed=19, views=nv)
    dc = torch.zeros_like(ds.color)
    dn = torch.zeros_like(ds.normal)
    dl = torch.zeros_like(ds.light_dir)
    dc_ref = np.zeros((sph.num_vertices, 3))
    dn_ref = np.zeros((sph.num_vertices, 3))
    dl_ref = np.zeros(3)
    gs = []
    for v in range(nv):
        sv = S.Scene(W, W, sph.pos, sph.tris, color=sph.color, normal=sph.normal, mvp=mvps[v],
                     light_dir=sph.light_dir, shade_mode=sph.shade_mode)
        ref_key, _ = oracle.raster_bbox(sv)
        assert_keys_equal(fbs[v].key_numpy(), ref_key, f"view {v}")
        g = np.zeros((W, W, 4))
        g[..., :3] = 2.0 * (oracle.shade(sv, ref_key)[..., :3] - tgt[v][..., :3])
        oracle.backward(sv, ref_key, g, out=(dc_ref, dn_ref, dl_ref))
        gs.append(torch.from_numpy(g.astype(np.float32)).cuda())
    r.backward_batch(views, fbs, gs, [dc] * nv, [dn] * nv, [dl] * nv)
    torch.cuda.synchronize()
    _grad_check(dc.cpu().numpy(), dc_ref)
    _grad_check(dn.cpu().numpy(), dn_ref)
    _grad_check(dl.cpu().numpy(), dl_ref)


# --------------------------------------------------------------- batches
def _batch_scenes(n, seed=0, small=True):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        side = int(rng.choice([64, 96, 128, 192])) if small else int(rng.choice(np.arange(256, 1025, 64)))
        T = int(rng.integers(50, 2000))
        kind = k % 3
        if kind == 0:
            s = S.random_triangles(side, side, T, float(rng.choice([3.0, 10.0, 40.0])), seed=int(rng.integers(1 << 30)),
                                   shade_mode=S.SHADE_GOURAUD)
        elif kind == 1:
            q = max(2, int(np.sqrt(T / 2)))
            s = S.heightfield(side, side, q, q, seed=int(rng.integers(1 << 30)), with_color=True)
        else:
            s = S.random_triangles(side, side + 32, T, 15.0, seed=int(rng.integers(1 << 30)),
                                   shade_mode=S.SHADE_LAMBERT, with_normals=True)
        out.append(s)
    return out


@pytest.mark.parametrize("launch", [0, 1])
def test_forward_batch_matches_oracle_and_single_scenes(launch):
    torch = _torch()
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene, Rasterizer
    scenes = _batch_scenes(12, seed=launch)
    bins = [(8, 8), (16, 16), (32, 32), (64, 64), (8, 32), (16, 64)] * 2
    sched = ["static", "dynamic"] * 6
    r = Rasterizer(64, 64, 16, 16)
    r.set_option(L.PIKO_OPT_BATCH_LAUNCH, launch)
    ds = [DeviceScene.from_host(s) for s in scenes]
    for rep in range(2):  # the second call reuses the zeroed counts and scan states
        fbs = r.forward_batch(ds, bin_sizes=bins, schedules=sched)
        torch.cuda.synchronize()
        assert r.status()[0] == 0
        for i, s in enumerate(scenes):
            ref, _ = oracle.raster_bbox(s)
            assert_keys_equal(fbs[i].key_numpy(), ref, f"batch scene {i} rep {rep}")
            assert np.abs(fbs[i].rgba.cpu().numpy() - oracle.shade(s, ref)).max() <= RGB_TOL


def test_forward_batch_gbuffer_and_empty_scenes():
    torch = _torch()
    from paper_1404_6293_gb300.raster import DeviceScene, Rasterizer
    a = S.power_law_triangles(160, 96, 3000, seed=3)
    b = S.Scene(40, 30, np.zeros((0, 4), np.float32), np.zeros((0, 3), np.int32), color=np.zeros((0, 3), np.float32))
    c = S.random_triangles(50, 70, 300, 8.0, seed=4)
    r = Rasterizer(64, 64)
    fbs = r.forward_batch([DeviceScene.from_host(x) for x in (a, b, c)], schedules=["dynamic", "static", "dynamic"])
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    ref_a, _ = oracle.raster_bbox(a)
    assert_keys_equal(fbs[0].key_numpy(), ref_a, "gbuffer scene")
    gn, ga = oracle.shade(a, ref_a)
    assert_half_close(fbs[0].gbuf_normal.cpu().numpy(), gn)
    assert (fbs[1].key_numpy() == EMPTY).all()
    ref_c, _ = oracle.raster_bbox(c)
    assert_keys_equal(fbs[2].key_numpy(), ref_c, "third scene")


def test_backward_batch_matches_single_scene_backward():
    torch = _torch()
    from paper_1404_6293_gb300.raster import DeviceScene, Rasterizer
    scenes = [s for s in _batch_scenes(6, seed=7) if s.shade_mode != S.SHADE_GBUFFER]
    ds = [DeviceScene.from_host(s) for s in scenes]
    r = Rasterizer(64, 64)
    fbs = r.forward_batch(ds)
    gs, dcs, dns, dls = [], [], [], []
    for i, s in enumerate(scenes):
        tgt = torch.from_numpy(S.target_image(s.width, s.height, seed=i)[0]).cuda()
        g = 2.0 * (fbs[i].rgba - tgt)
        g[..., 3] = 0
        gs.append(g.contiguous())
        dcs.append(torch.zeros((s.num_vertices, 3), device="cuda"))
        dns.append(torch.zeros((s.num_vertices, 3), device="cuda") if s.normal is not None else None)
        dls.append(torch.zeros(3, device="cuda"))
    r.backward_batch(ds, fbs, gs, dcs, dns, dls)
    torch.cuda.synchronize()
    for i, s in enumerate(scenes):
        ref_key, _ = oracle.raster_bbox(s)
        g = gs[i].cpu().numpy().astype(np.float64)
        dc, dn, dl = oracle.backward(s, ref_key, g)
        _grad_check(dcs[i].cpu().numpy(), dc)
        if s.shade_mode == S.SHADE_LAMBERT:
            _grad_check(dns[i].cpu().numpy(), dn)
            _grad_check(dls[i].cpu().numpy(), dl)
