"""The exact triangle-vs-bin overlap test of AssignBin (PIKO_OPT_EXACT_BINS),
checked on the CPU against what it must guarantee.

- It is conservative: a bin in which the oracle finds a covered pixel of a
  triangle (the triangle rendered alone, so nothing hides it) is never
  dropped; and it keeps only bins of the bounding box.
- It is tight where the answer is known by hand: a right triangle over a
  64x64 frame of 8x8 bins keeps exactly the 36 bins its hypotenuse does not
  leave behind.
The GPU's counts are compared with this model in tests/test_gpu_exact_bins.py.
"""
import numpy as np

import oracle
from binning_model import kept_bins
from paper_1404_6293_gb300 import scenes as S

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


def _one(W, H, px, py):
    """A one-triangle scene with vertices at pixel coordinates (px[i], py[i])."""
    px, py = np.asarray(px, float), np.asarray(py, float)
    pos = np.stack([px / W * 2 - 1, 1 - py / H * 2, np.zeros(3), np.ones(3)], 1).astype(np.float32)
    return S.Scene(W, H, pos, np.arange(3, dtype=np.int32).reshape(1, 3),
                   color=np.ones((3, 3), np.float32), name="one")


def _snapped(scene):
    X, Y, _, ok = oracle.vertex_stage(scene)
    assert ok.all()
    return [(int(X[i]), int(Y[i])) for i in range(3)]


def test_hand_derived_right_triangle_keeps_36_of_64_bins():
    # vertices (0, 0), (64, 0), (0, 64): covered centres (a + 1/2, b + 1/2)
    # with a + b <= 62 (a + b + 1 < 64; on the hypotenuse a + b = 63 the
    # fill rule decides).  Bin (bx, by) has centres with a + b >= 8 (bx + by),
    # so it holds covered centres exactly when bx + by <= 7: 36 of the 64.
    s = _one(64, 64, [0, 64, 0], [0, 0, 64])
    kept, box = kept_bins(_snapped(s), 64, 64, 8, 8)
    assert len(box) == 64
    assert sorted(kept) == sorted((bx, by) for by in range(8) for bx in range(8) if bx + by <= 7)
    # and it agrees with the oracle's coverage of the same triangle
    key, _ = oracle.raster_bbox(s)
    hit = {(int(x) // 8, int(y) // 8) for y, x in np.argwhere(key != EMPTY)}
    assert hit == set(kept)


def test_kept_bins_cover_every_covered_pixel_and_stay_in_the_box():
    rng = np.random.default_rng(20261205)
    W, H = 160, 112
    checked = dropped = 0
    for trial in range(300):
        kind = trial % 3
        c = rng.uniform([0.1 * W, 0.1 * H], [0.9 * W, 0.9 * H])
        if kind == 0:    # long and thin, any angle
            ang = rng.uniform(0, np.pi)
            d = np.array([np.cos(ang), np.sin(ang)]) * rng.uniform(20, 150)
            n = np.array([-d[1], d[0]]) / np.linalg.norm(d) * rng.uniform(0.3, 4.0)
            P = np.array([c - d / 2, c + d / 2, c + n])
        elif kind == 1:  # large, random
            P = c + rng.uniform(-80, 80, (3, 2))
        else:            # small
            P = c + rng.uniform(-6, 6, (3, 2))
        s = _one(W, H, P[:, 0], P[:, 1])
        X, Y, _, ok = oracle.vertex_stage(s)
        if not ok.all():
            continue
        key, _ = oracle.raster_bbox(s)
        covered = np.argwhere(key != EMPTY)
        for bw, bh in ((8, 8), (16, 16), (32, 8)):
            kept, box = kept_bins([(int(X[i]), int(Y[i])) for i in range(3)], W, H, bw, bh)
            hit = {(int(x) // bw, int(y) // bh) for y, x in covered}
            assert hit <= set(kept), (trial, bw, bh, sorted(hit - set(kept)))
            assert set(kept) <= set(box)
            checked += 1
            dropped += len(box) - len(kept)
    assert checked > 800 and dropped > 0  # the test does drop bins
