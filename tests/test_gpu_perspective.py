"""Perspective-correct attributes (PIKO_OPT_PERSPECTIVE) on the GPU against
the oracle's O15 reading, through the C ABI.

Coverage and depth do not change with the option, so keys must stay
bit-exact. Colours must be within 1e-5 absolute of the float64 oracle, and
binary16 G-buffer values within one step. Gradients must be within 1e-4
relative, as in the screen-space tests. The scenes come with real
perspective cameras, so w varies across each triangle. They cover:
- the per-thread and per-warp coverage paths;
- shading from records, and from global memory when a tile's records run out;
- both backward forms.
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


def _sphere(W, H, slices, stacks, mode, seed=11):
    sph, mvps = S.sphere_views(num_views=1, width=W, height=H, slices=slices, stacks=stacks, seed=seed)
    sph.shade_mode = mode
    sph.mvp = np.ascontiguousarray(mvps[0], np.float32).reshape(16)
    return sph


def _floor(W=128, H=96):
    world = np.array([[-1.5, 0.0, -0.5], [1.5, 0.0, -0.5], [1.5, 0.0, -6.0], [-1.5, 0.0, -6.0]])
    tris = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    M = S._look_at_perspective([0.0, 1.0, 1.0], [0.0, 0.0, -3.0], [0.0, 1.0, 0.0], 60.0, W / H, 0.1, 20.0)
    color = world @ np.array([[0.25, 0.0, 0.05], [0.0, 0.0, -0.15], [0.1, 0.0, 0.1]]).T + [0.5, 0.1, 0.8]
    pos = np.concatenate([world, np.ones((4, 1))], 1).astype(np.float32)
    return S.Scene(W, H, pos, tris, color=color.astype(np.float32), mvp=M.astype(np.float32).reshape(16))


def _render(scene, bins=16, schedule="hardware", perspective=True, extra=None):
    torch = _torch()
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene, Rasterizer
    r = Rasterizer(scene.width, scene.height, bins, bins, schedule)
    r.set_option(L.PIKO_OPT_PERSPECTIVE, 1 if perspective else 0)
    for k, v in (extra or {}).items():
        r.set_option(k, v)
    ds = DeviceScene.from_host(scene)
    fb = r.forward(ds)
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    return r, ds, fb


def _check_colour(scene, fb, ref_key, check_differs=True):
    if scene.shade_mode == S.SHADE_GBUFFER:
        gn, ga = oracle.shade(scene, ref_key, perspective=True)
        for got, ref in ((fb.gbuf_normal, gn), (fb.gbuf_albedo, ga)):
            g = got.cpu().numpy().astype(np.float64)
            r = ref.view(np.float16).astype(np.float64)
            step = np.spacing(np.maximum(np.abs(g), np.abs(r)).astype(np.float16)).astype(np.float64)
            assert np.all(np.abs(g - r) <= step)
        return
    rgba_ref = oracle.shade(scene, ref_key, perspective=True)
    err = np.abs(fb.rgba.cpu().numpy() - rgba_ref).max()
    assert err <= RGB_TOL, err
    if check_differs:  # the option matters on this scene
        assert np.abs(oracle.shade(scene, ref_key)[..., :3] - rgba_ref[..., :3]).max() > 100 * RGB_TOL


@pytest.mark.parametrize("mode", [S.SHADE_GOURAUD, S.SHADE_LAMBERT, S.SHADE_GBUFFER])
@pytest.mark.parametrize("schedule", ["static", "dynamic", "hardware"])
def test_sphere_view_matches_oracle(mode, schedule):
    s = _sphere(192, 160, 48, 32, mode)
    ref_key, _ = oracle.raster_bbox(s)
    _, _, fb = _render(s, 16, schedule)
    assert np.array_equal(fb.key_numpy(), ref_key)
    _check_colour(s, fb, ref_key)


@pytest.mark.parametrize("bins", [16, 32])
def test_large_triangles_take_the_warp_path(bins):
    from paper_1404_6293_gb300 import _lib as L
    s = _floor()
    ref_key, _ = oracle.raster_brute(s)
    for small_px in (1, 4096):  # every box by a warp, then every box by one thread
        _, _, fb = _render(s, bins, "dynamic", extra={L.PIKO_OPT_SMALL_TRI_PIXELS: small_px})
        assert np.array_equal(fb.key_numpy(), ref_key)
        _check_colour(s, fb, ref_key)


def test_tiles_past_their_records_shade_from_global_memory():
    # 99.5k triangles over 8x8 tiles of 16x16 pixels: far more entries per
    # tile than shading records, so most winners are shaded from global memory
    s = _sphere(128, 128, 250, 200, S.SHADE_LAMBERT)
    ref_key, _ = oracle.raster_bbox(s, threads=8)
    _, _, fb = _render(s, 16, "hardware")
    assert np.array_equal(fb.key_numpy(), ref_key)
    _check_colour(s, fb, ref_key, check_differs=False)


def _grad_check(g_gpu, g_ref):
    g_gpu = np.asarray(g_gpu, np.float64)
    scale = np.abs(g_ref).max()
    big = np.abs(g_ref) > 1e-3 * scale
    assert scale > 0
    rel = np.abs(g_gpu - g_ref)[big] / np.abs(g_ref)[big]
    assert rel.max() <= 1e-4, rel.max()
    assert np.abs(g_gpu - g_ref)[~big].max(initial=0) <= 1e-4 * scale


@pytest.mark.parametrize("form", ["tile", "pixel"])
@pytest.mark.parametrize("mode", [S.SHADE_GOURAUD, S.SHADE_LAMBERT])
def test_backward_forms_match_oracle(form, mode):
    torch = _torch()
    if form == "tile":
        s = _sphere(192, 160, 40, 30, mode)
        assert 4 * s.num_triangles <= s.width * s.height
    else:
        s = _sphere(96, 80, 60, 40, mode)
        assert 4 * s.num_triangles > s.width * s.height
    r, ds, fb = _render(s, 16, "dynamic")
    ref_key, _ = oracle.raster_bbox(s)
    assert np.array_equal(fb.key_numpy(), ref_key)
    tgt = S.target_image(s.width, s.height, seed=6)[0]
    g = np.zeros((s.height, s.width, 4))
    g[..., :3] = 2.0 * (oracle.shade(s, ref_key, perspective=True)[..., :3] - tgt[..., :3])
    dc, dn, dl = oracle.backward(s, ref_key, g, perspective=True)
    V = s.num_vertices
    dcg = torch.zeros((V, 3), device="cuda")
    dng = torch.zeros((V, 3), device="cuda")
    dlg = torch.zeros(3, device="cuda")
    r.backward(ds, fb, torch.from_numpy(g.astype(np.float32)).cuda(), dcg, dng, dlg)
    torch.cuda.synchronize()
    _grad_check(dcg.cpu().numpy(), dc)
    if mode == S.SHADE_LAMBERT:
        _grad_check(dng.cpu().numpy(), dn)
        _grad_check(dlg.cpu().numpy(), dl)


def test_batch_with_the_option_equals_single_scene_calls():
    """Perspective and unclamped shading in a batch: every scene's keys,
    colours and gradients as its single-scene call gives them."""
    torch = _torch()
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene, Rasterizer
    host = [_sphere(160, 128, 40, 30, S.SHADE_LAMBERT, seed=3), _floor(128, 96),
            _sphere(96, 80, 60, 40, S.SHADE_GOURAUD, seed=4)]
    for opts in ({L.PIKO_OPT_PERSPECTIVE: 1}, {L.PIKO_OPT_PERSPECTIVE: 1, L.PIKO_OPT_UNCLAMPED: 1},
                 {L.PIKO_OPT_UNCLAMPED: 1}):
        ds = [DeviceScene.from_host(s) for s in host]
        rb = Rasterizer(64, 64)
        for k, v in opts.items():
            rb.set_option(k, v)
        fbs = rb.forward_batch(ds, None, [(16, 16), (32, 32), (16, 16)], ["dynamic", "static", "dynamic"])
        torch.cuda.synchronize()
        assert rb.status()[0] == 0
        grads_b, grads_s = [], []
        gl = []
        for i, s in enumerate(host):
            tgt = torch.from_numpy(S.target_image(s.width, s.height, seed=9 + i)[0]).cuda()
            gl.append((2.0 * (fbs[i].rgba - tgt)).contiguous())
            gl[-1][..., 3] = 0
            grads_b.append([torch.zeros((s.num_vertices, 3), device="cuda"), torch.zeros((s.num_vertices, 3),
                            device="cuda"), torch.zeros(3, device="cuda")])
        rb.backward_batch(ds, fbs, gl, [g[0] for g in grads_b], [g[1] if s.normal is not None else None
                                                                  for g, s in zip(grads_b, host)],
                          [g[2] if s.normal is not None else None for g, s in zip(grads_b, host)])
        torch.cuda.synchronize()
        assert rb.status()[0] == 0
        for i, s in enumerate(host):
            r = Rasterizer(s.width, s.height, 16, 16, "hardware")
            for k, v in opts.items():
                r.set_option(k, v)
            fb = r.forward(ds[i])
            torch.cuda.synchronize()
            assert torch.equal(fb.key, fbs[i].key), f"scene {i} keys"
            assert (fb.rgba - fbs[i].rgba).abs().max().item() <= 1e-6, f"scene {i} colours"
            ref_key, _ = oracle.raster_bbox(s)
            persp = bool(opts.get(L.PIKO_OPT_PERSPECTIVE, 0))
            unc = bool(opts.get(L.PIKO_OPT_UNCLAMPED, 0))
            ref = oracle.shade(s, ref_key, perspective=persp, unclamped=unc)
            assert np.abs(fbs[i].rgba.cpu().numpy() - ref).max() <= RGB_TOL
            g = [torch.zeros_like(t) for t in grads_b[i]]
            r.backward(ds[i], fb, gl[i], g[0], g[1] if s.normal is not None else None,
                       g[2] if s.normal is not None else None)
            torch.cuda.synchronize()
            _grad_check(grads_b[i][0].cpu().numpy(), g[0].cpu().numpy().astype(np.float64))
            if s.shade_mode == S.SHADE_LAMBERT:  # Gouraud has no normal or light gradients
                _grad_check(grads_b[i][1].cpu().numpy(), g[1].cpu().numpy().astype(np.float64))
                _grad_check(grads_b[i][2].cpu().numpy(), g[2].cpu().numpy().astype(np.float64))
            r.close()
        rb.close()


def test_option_after_reserve_needs_no_allocation_in_a_graph():
    """reserve() sizes the 1/w buffer too, so a forward captured in a CUDA
    graph after turning the option on allocates nothing."""
    torch = _torch()
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene, Framebuffer, Rasterizer
    s = _sphere(128, 96, 24, 16, S.SHADE_LAMBERT)
    r = Rasterizer(s.width, s.height, 16, 16, "hardware")
    ds = DeviceScene.from_host(s)
    fb = Framebuffer.allocate(s.width, s.height, s.shade_mode)
    r.reserve(s.num_vertices, s.num_triangles, 1 << 20)
    r.set_option(L.PIKO_OPT_CHECK_CAPACITY, 0)
    r.set_option(L.PIKO_OPT_PERSPECTIVE, 1)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        r.forward(ds, fb, side)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        r.forward(ds, fb)
    fb.key.fill_(0)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    ref_key, _ = oracle.raster_bbox(s)
    assert np.array_equal(fb.key_numpy(), ref_key)
    assert np.abs(fb.rgba.cpu().numpy() - oracle.shade(s, ref_key, perspective=True)).max() <= RGB_TOL
    r.close()
