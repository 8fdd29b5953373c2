"""Bounded device-side waits that run out are reported, not hung on.

The look-back scan and the batch kernel's grid barrier wait on other CTAs
with a clock budget (PIKO_OPT_WAIT_BUDGET).  The test hook
PIKO_OPT_TEST_WITHHOLD keeps one publication from happening -- scan chunk 0's
prefix, or CTA 0's arrival at the first grid barrier -- so that a wait has
nothing to wait for and runs out; nothing faults.  The frame must report
PIKO_ERR_TIMEOUT, leave its output untouched (the later phases skip their
work), and the next frame without the hook must be exact again.
"""
import numpy as np
import pytest

import oracle
from paper_1404_6293_gb300 import scenes as S

pytestmark = pytest.mark.gpu

SHORT_BUDGET_KCYCLES = 20  # 20,000 SM cycles: about 10 us


def _torch():
    import torch
    return torch


def test_scan_wait_runs_out_and_reports_timeout():
    torch = _torch()
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene, Framebuffer, Rasterizer
    s = S.random_triangles(1024, 1024, 4000, 12.0, seed=91)  # 128 x 128 = 16384 tiles: eight scan chunks
    r = Rasterizer(s.width, s.height, 8, 8, "dynamic")
    ds = DeviceScene.from_host(s)
    fb = Framebuffer.allocate(s.width, s.height, s.shade_mode)
    r.forward(ds, fb)
    assert r.status()[0] == L.PIKO_OK
    r.set_option(L.PIKO_OPT_CHECK_CAPACITY, 0)
    r.set_option(L.PIKO_OPT_WAIT_BUDGET, SHORT_BUDGET_KCYCLES)
    r.set_option(L.PIKO_OPT_TEST_WITHHOLD, 1)
    fb.key.fill_(1234)
    fb.rgba.fill_(3.0)
    r.forward(ds, fb)
    torch.cuda.synchronize()
    assert r.status()[0] == L.PIKO_ERR_TIMEOUT
    assert bool((fb.key == 1234).all()) and bool((fb.rgba == 3.0).all()), "a timed-out frame wrote output"
    # the status word is cleared by the read; the next frame is exact
    r.set_option(L.PIKO_OPT_TEST_WITHHOLD, 0)
    r.set_option(L.PIKO_OPT_WAIT_BUDGET, 40000)
    r.forward(ds, fb)
    torch.cuda.synchronize()
    assert r.status()[0] == L.PIKO_OK
    ref, _ = oracle.raster_bbox(s, threads=8)
    assert np.array_equal(fb.key_numpy(), ref)


@pytest.mark.parametrize("withhold", [1, 2])
def test_batch_waits_run_out_and_report_timeout(withhold):
    """withhold 1: the batch scan's chunk 0 keeps its prefix; 2: CTA 0 never
    arrives at the first grid barrier, so every CTA's barrier wait runs out."""
    torch = _torch()
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene, Rasterizer
    host = [S.random_triangles(512, 512, 2000, 10.0, seed=92 + i) for i in range(3)]  # 3 x 1024 tiles
    ds = [DeviceScene.from_host(h) for h in host]
    n = len(ds)
    bins, scheds = [(16, 16)] * n, ["dynamic"] * n
    r = Rasterizer(64, 64, 16, 16)
    fbs = r.forward_batch(ds, None, bins, scheds)
    torch.cuda.synchronize()
    assert r.status()[0] == L.PIKO_OK
    r.set_option(L.PIKO_OPT_CHECK_CAPACITY, 0)
    r.set_option(L.PIKO_OPT_WAIT_BUDGET, SHORT_BUDGET_KCYCLES)
    r.set_option(L.PIKO_OPT_TEST_WITHHOLD, withhold)
    for f in fbs:
        f.key.fill_(1234)
    r.forward_batch(ds, fbs, bins, scheds)
    torch.cuda.synchronize()
    assert r.status()[0] == L.PIKO_ERR_TIMEOUT
    for i, f in enumerate(fbs):
        assert bool((f.key == 1234).all()), f"scene {i}: a timed-out batch wrote keys"
    r.set_option(L.PIKO_OPT_TEST_WITHHOLD, 0)
    r.set_option(L.PIKO_OPT_WAIT_BUDGET, 40000)
    r.forward_batch(ds, fbs, bins, scheds)
    torch.cuda.synchronize()
    assert r.status()[0] == L.PIKO_OK
    for i in range(n):
        ref, _ = oracle.raster_bbox(host[i], threads=8)
        assert np.array_equal(fbs[i].key_numpy(), ref), f"scene {i} after the timed-out batch"
