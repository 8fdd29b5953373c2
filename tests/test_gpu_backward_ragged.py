"""Backward parity on image sizes that are not multiples of the 16 x 16
backward tile, so that every tile row and column has a ragged tail: the
tile form (a warp per tile, runs down each lane's column), the per-pixel
form and the batch kernel, each against the oracle's float64 gradients
(the attribute gradients of the Lambert shader of Listing 1 and of Gouraud
interpolation, visibility fixed by the forward keys)."""
import numpy as np
import pytest

import oracle
from paper_1404_6293_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _grad_check(g_gpu, g_ref):
    g_gpu = np.asarray(g_gpu, np.float64)
    scale = np.abs(g_ref).max()
    assert scale > 0
    big = np.abs(g_ref) > 1e-3 * scale
    rel = np.abs(g_gpu - g_ref)[big] / np.abs(g_ref)[big]
    assert rel.max() <= 1e-4, rel.max()
    assert np.abs(g_gpu - g_ref)[~big].max(initial=0) <= 1e-4 * scale


def _loss_grad(s, ref_key, seed):
    tgt = S.target_image(s.width, s.height, seed=seed)[0]
    g = np.zeros((s.height, s.width, 4))
    if s.shade_mode != S.SHADE_GBUFFER:
        g[..., :3] = 2.0 * (oracle.shade(s, ref_key)[..., :3] - tgt[..., :3])
    return g


def _single(s, seed):
    torch = _torch()
    from paper_1404_6293_gb300.raster import DeviceScene, Rasterizer
    r = Rasterizer(s.width, s.height, 16, 16, "dynamic")
    ds = DeviceScene.from_host(s)
    fb = r.forward(ds)
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    ref_key, _ = oracle.raster_brute(s)
    assert np.array_equal(fb.key_numpy(), ref_key)
    g = _loss_grad(s, ref_key, seed)
    V = s.num_vertices
    dc = torch.zeros((V, 3), device="cuda")
    dn = torch.zeros((V, 3), device="cuda")
    dl = torch.zeros(3, device="cuda")
    r.backward(ds, fb, torch.from_numpy(g.astype(np.float32)).cuda(), dc, dn, dl)
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    rc, rn, rl = oracle.backward(s, ref_key, g)
    if s.shade_mode == S.SHADE_GOURAUD or s.color is not None:
        _grad_check(dc.cpu().numpy(), rc)
    if s.shade_mode == S.SHADE_LAMBERT:
        _grad_check(dn.cpu().numpy(), rn)
        _grad_check(dl.cpu().numpy(), rl)
    r.close()


@pytest.mark.parametrize("W,H", [(150, 101), (33, 17), (47, 9)])
def test_tile_form_ragged_lambert(W, H):
    # large triangles (at most one per four pixels): the tile form
    s = S.random_triangles(W, H, max(4, W * H // 60), 0.35 * max(W, H), seed=W + H,
                           shade_mode=S.SHADE_LAMBERT, with_normals=True)
    s.light_dir = np.array([0.3, -0.4, -0.866], np.float32)
    assert 4 * s.num_triangles <= W * H
    _single(s, seed=3)


def test_tile_form_ragged_gouraud_one_run_per_column():
    # two triangles covering the whole 70 x 37 image: every lane's column is
    # one run per tile, flushed once at the tile's (ragged) end
    W, H = 70, 37
    pos = np.array([[-1, -1, 0.2, 1], [1, -1, 0.4, 1], [1, 1, 0.6, 1], [-1, 1, 0.3, 1]], np.float32)
    tris = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    col = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0]], np.float32)
    s = S.Scene(W, H, pos, tris, color=col, shade_mode=S.SHADE_GOURAUD)
    _single(s, seed=4)


def test_pixel_form_ragged():
    # tiny triangles (more than one per four pixels): the per-pixel form
    s = S.heightfield(97, 61, 50, 40, seed=79, shade_mode=S.SHADE_LAMBERT, with_color=True)
    assert 4 * s.num_triangles > s.width * s.height
    _single(s, seed=6)


def test_batch_backward_ragged_scenes():
    torch = _torch()
    from paper_1404_6293_gb300.raster import DeviceScene, Rasterizer
    scenes = [
        S.random_triangles(150, 101, 300, 30.0, seed=81, shade_mode=S.SHADE_LAMBERT, with_normals=True),
        S.random_triangles(77, 45, 120, 9.0, seed=82, shade_mode=S.SHADE_GOURAUD),
        S.heightfield(200, 33, 40, 8, seed=83, shade_mode=S.SHADE_LAMBERT, with_color=True),
        S.random_triangles(31, 129, 900, 3.0, seed=84, shade_mode=S.SHADE_LAMBERT, with_normals=True),
    ]
    for s in scenes:
        s.light_dir = np.array([-0.2, 0.5, -0.84], np.float32)
    ds = [DeviceScene.from_host(s) for s in scenes]
    r = Rasterizer(64, 64)
    fbs = r.forward_batch(ds, None, [(16, 16)] * len(scenes), ["dynamic"] * len(scenes))
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    gs, dcs, dns, dls, refs = [], [], [], [], []
    for i, s in enumerate(scenes):
        ref_key, _ = oracle.raster_brute(s)
        assert np.array_equal(fbs[i].key_numpy(), ref_key), i
        g = _loss_grad(s, ref_key, seed=10 + i)
        refs.append((ref_key, g))
        gs.append(torch.from_numpy(g.astype(np.float32)).cuda())
        dcs.append(torch.zeros((s.num_vertices, 3), device="cuda"))
        dns.append(torch.zeros((s.num_vertices, 3), device="cuda") if s.normal is not None else None)
        dls.append(torch.zeros(3, device="cuda"))
    r.backward_batch(ds, fbs, gs, dcs, dns, dls)
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    for i, s in enumerate(scenes):
        ref_key, g = refs[i]
        rc, rn, rl = oracle.backward(s, ref_key, g)
        if s.shade_mode == S.SHADE_GOURAUD or s.color is not None:
            _grad_check(dcs[i].cpu().numpy(), rc)
        if s.shade_mode == S.SHADE_LAMBERT:
            _grad_check(dns[i].cpu().numpy(), rn)
            _grad_check(dls[i].cpu().numpy(), rl)
    r.close()
