"""The autotuner: workload classes and the cache on CPU; on the GPU, that its
choices are valid knobs and that rendering with them still matches the
oracle (the tuner only ever picks among settings that cannot change output)."""
import json

import numpy as np
import pytest
import torch

from paper_1404_6293_gb300 import scenes as S
from paper_1404_6293_gb300.autotune import (BATCH_SCHEDULES, DEFAULT_BINS, DEFAULT_SCHEDULES, OTHER_MAPPINGS,
                                            THREAD_CHOICES,
                                            Autotuner, default_threads, features, thread_candidates)
from paper_1404_6293_gb300.raster import DeviceScene


def _cpu_scene(W, H, T, mode=S.SHADE_LAMBERT):
    # a DeviceScene with CPU tensors: features() only reads sizes and mode
    return DeviceScene(W, H, torch.zeros((3 * T, 4)), torch.zeros((T, 3), dtype=torch.int32), None, None, None,
                       None, mode)


def test_features_bucket_sizes_density_and_mode():
    a = features(_cpu_scene(1920, 1080, 1_000_000))
    assert a == features(_cpu_scene(1920, 1080, 1_050_000))  # same class: within a half-octave bucket
    assert a != features(_cpu_scene(1920, 1080, 250_000))    # fewer triangles, lower density
    assert a != features(_cpu_scene(960, 540, 1_000_000))     # fewer pixels
    assert a != features(_cpu_scene(1920, 1080, 1_000_000, S.SHADE_GBUFFER))


def test_cache_round_trip_answers_without_measuring(tmp_path):
    scene = _cpu_scene(512, 512, 20_000)
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({features(scene): {"bin": [32, 32], "schedule": "dynamic", "ms": 1.0}}))
    tuner = Autotuner(cache_path=str(path))
    # a cached class needs no GPU: choose() answers from the cache
    assert tuner.choose(scene) == ((32, 32), "dynamic")
    tuner.save(str(tmp_path / "copy.json"))
    assert json.loads((tmp_path / "copy.json").read_text()) == json.loads(path.read_text())


def test_thread_candidates_around_the_library_default():
    # the library's defaults (piko_internal.cuh): 64 up to 64 pixels, 128 up to 256, else 256
    assert [default_threads(b * b) for b in (8, 16, 32, 64)] == [64, 128, 256, 256]
    for b in (8, 16, 32, 64):
        c = thread_candidates(b, b)
        assert default_threads(b * b) in c
        assert all(t in THREAD_CHOICES and t <= max(64, b * b) for t in c)
    assert thread_candidates(16, 16) == (64, 128, 256)
    assert thread_candidates(8, 8) == (64,)


def test_cached_entry_without_threads_uses_the_default(tmp_path):
    scene = _cpu_scene(640, 480, 50_000)
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({features(scene): {"bin": [16, 16], "schedule": "hardware", "ms": 1.0}}))
    tuner = Autotuner(cache_path=str(path))
    assert tuner.knobs(scene) == {"bin": (16, 16), "schedule": "hardware", "threads": 128, "exact_bins": 0}
    path.write_text(json.dumps({features(scene): {"bin": [32, 32], "schedule": "static", "threads": 512,
                                                  "ms": 1.0}}))
    assert Autotuner(cache_path=str(path)).knobs(scene)["threads"] == 512


def test_batch_candidates_exclude_the_hardware_mapping():
    assert "hardware" in DEFAULT_SCHEDULES
    assert "hardware" not in BATCH_SCHEDULES


@pytest.mark.gpu
def test_tuned_settings_are_valid_and_render_exactly():
    import oracle
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import Rasterizer
    host = S.scene_batch(6, tmax=20_000, side_max=384, seed=5)
    ds = [DeviceScene.from_host(s) for s in host]
    tuner = Autotuner(bins=((16, 16), (32, 32)), reps=1)
    k = tuner.knobs(ds[0])
    (bw, bh), sched = tuner.choose(ds[0])
    assert (bw, bh) == k["bin"] and sched == k["schedule"]
    assert (bw, bh) in ((16, 16), (32, 32)) and sched in DEFAULT_SCHEDULES + OTHER_MAPPINGS
    assert k["threads"] in thread_candidates(bw, bh) or sched in OTHER_MAPPINGS
    # every candidate was timed: bins x schedules x threads, plus the two other mappings
    trials = next(iter(tuner.cache.values()))["trials"]
    assert {t["schedule"] for t in trials} == set(DEFAULT_SCHEDULES + OTHER_MAPPINGS)
    # the best binned candidate was also timed with exact bins
    assert sum(1 for t in trials if t.get("exact_bins")) == 1
    # the tuned knobs render the scene exactly
    r1 = Rasterizer(host[0].width, host[0].height, bw, bh, sched)
    r1.set_option(L.PIKO_OPT_THREADS_PER_TILE, k["threads"])
    r1.set_option(L.PIKO_OPT_EXACT_BINS, k["exact_bins"])
    fb1 = r1.forward(ds[0])
    torch.cuda.synchronize()
    assert r1.status()[0] == 0
    assert np.array_equal(fb1.key_numpy(), oracle.raster_bbox(host[0])[0])
    r1.close()
    bins, scheds, report = tuner.tune_batch(ds)
    tuner.close()
    assert len(bins) == len(scheds) == len(ds)
    assert report["choice"] in ("uniform", "per_class")
    assert all(tuple(b) in ((16, 16), (32, 32)) for b in bins) and all(s in BATCH_SCHEDULES for s in scheds)
    r = Rasterizer(64, 64)
    fbs = r.forward_batch(ds, None, bins, scheds)
    torch.cuda.synchronize()
    assert r.status()[0] == 0
    for i, s in enumerate(host):
        ref, _ = oracle.raster_bbox(s)
        assert np.array_equal(fbs[i].key_numpy(), ref), f"scene {i}"


@pytest.mark.gpu
def test_render_from_host_equals_forward():
    from paper_1404_6293_gb300.raster import Framebuffer, Rasterizer
    s = S.heightfield(320, 200, 60, 40, seed=8)
    ds = DeviceScene.from_host(s)
    r = Rasterizer(s.width, s.height, 16, 16, "hardware")
    fb = r.forward(ds)
    torch.cuda.synchronize()
    ref_key, ref_rgba = fb.key.cpu(), fb.rgba.cpu()
    names = [n for n in ("pos", "tris", "normal", "color", "mvp", "light_dir") if getattr(ds, n) is not None]
    host_in = {n: getattr(ds, n).cpu().pin_memory() for n in names}
    ds2 = DeviceScene.from_host(s)
    for n in names:
        getattr(ds2, n).zero_()  # the copies must bring the inputs back
    fb2 = Framebuffer.allocate(s.width, s.height, s.shade_mode)
    key_h = torch.empty_like(fb2.key, device="cpu").pin_memory()
    rgba_h = torch.empty_like(fb2.rgba, device="cpu").pin_memory()
    side = torch.cuda.Stream()
    r.render_from_host(host_in, ds2, fb2, key_h, rgba_h, stream=side)
    side.synchronize()
    assert torch.equal(key_h, ref_key) and torch.equal(rgba_h, ref_rgba)
