"""The Reyes Sample stage (Sec. 7.1 of the Piko paper) on this path:
micropolygon grids, as a Dice stage emits them, sampled at pixel centres
through the same AssignBin (bounding-box bins) and Process as the raster
pipeline, with the Sample stage's 32 x 32 bins and a diffuse Shade.  Keys
bit-exact and colours within 1e-5 of the oracle."""
import numpy as np
import pytest

import oracle
from paper_1404_6293_gb300 import scenes as S

pytestmark = pytest.mark.gpu

RGB_TOL = 1e-5


@pytest.mark.parametrize("bins,schedule", [(32, "dynamic"), (32, "static"), (32, "hardware"), (16, "hardware")])
def test_micropolygon_grids_sampled_exactly(bins, schedule):
    import torch
    from paper_1404_6293_gb300.raster import DeviceScene, Rasterizer
    s = S.reyes_grids(256, 192, 12, seed=5, side_max=64.0)
    ref, st = oracle.raster_bbox(s, threads=8)
    assert st == 0 and (ref != oracle.KEY_EMPTY).sum() > 0.2 * s.width * s.height
    r = Rasterizer(s.width, s.height, bins, bins, schedule)
    fb = r.forward(DeviceScene.from_host(s))
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    got = fb.key_numpy()
    bad = np.argwhere(got != ref)
    assert bad.size == 0, f"{len(bad)} keys differ, first at {tuple(bad[0][::-1])}"
    assert np.abs(fb.rgba.cpu().numpy() - oracle.shade(s, ref)).max() <= RGB_TOL


def test_micropolygon_grids_full_size_32x32_bins():
    """The bench's Sample workload (256 patches at 1024 x 768, 32 x 32 bins,
    dynamic schedule): every key bit-exact and every colour within 1e-5."""
    import torch
    from paper_1404_6293_gb300.raster import DeviceScene, Rasterizer
    s = S.reyes_grids()
    ref, _ = oracle.raster_bbox(s, threads=16)
    r = Rasterizer(s.width, s.height, 32, 32, "dynamic")
    fb = r.forward(DeviceScene.from_host(s))
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    assert np.array_equal(fb.key_numpy(), ref)
    assert np.abs(fb.rgba.cpu().numpy() - oracle.shade(s, ref)).max() <= RGB_TOL
