"""Autotuner for the binning and scheduling knobs.

The Piko paper explores bin size and schedule by hand for each scene and
architecture (Sec. 7.2: spatial binning helps most scenes but not one made
of tiny uniform triangles; fusing stages trades load balance for locality).
This tuner searches the same knobs automatically: for a scene it times the
forward pass under every (bin size, schedule, threads per bin) candidate with
CUDA events and keeps the fastest; the fused (no tiling) and unfused (one
kernel per stage) mappings of Sec. 7.2 are two more candidates, and the best binned candidate is
timed once more with AssignBin's exact overlap test (PIKO_OPT_EXACT_BINS) instead of bounding-box
bins, which pays for large and thin triangles.  Threads per bin is the third template
parameter of the paper's Listing 1 stage; small triangles favour fewer
threads per bin (more CTAs per SM), large ones more (more warps per tile).  Results are cached by workload features (resolution,
triangle count, coverage density, shading mode) so that similar scenes share
one measurement; the cache can be saved to and loaded from JSON.

A choice that is best for a scene rendered alone need not be best inside a
batch, where all scenes share one persistent launch (there is no per-scene
launch or grid-size effect).  ``tune_batch`` therefore measures inside the
batched pass itself: every workload class is timed as a sub-batch under each
candidate, and the assembled per-class choice is kept only if the whole batch
then beats the best uniform setting.
"""
from __future__ import annotations

import json
import math
import os
from typing import Dict, Iterable, List, Optional, Tuple

import torch

from . import _lib as L
from .raster import DeviceScene, Rasterizer

DEFAULT_BINS: Tuple[Tuple[int, int], ...] = ((8, 8), (16, 16), (32, 32), (64, 64))
DEFAULT_SCHEDULES: Tuple[str, ...] = ("static", "dynamic", "hardware")
THREAD_CHOICES: Tuple[int, ...] = (64, 128, 256, 512)  # the CTA sizes the library accepts
# a batch has no hardware mapping (its tiles are dealt inside one persistent launch)
BATCH_SCHEDULES: Tuple[str, ...] = ("static", "dynamic")
# the other two mappings of the pipeline (no tiling; one kernel per stage):
# bin size and threads per bin do not apply, so each is one candidate
OTHER_MAPPINGS: Tuple[str, ...] = ("fused", "unfused")


def default_threads(bin_px: int) -> int:
    """The library's CTA size for a bin of bin_px pixels when none is set."""
    return 64 if bin_px <= 64 else (128 if bin_px <= 256 else 256)


def thread_candidates(bw: int, bh: int) -> Tuple[int, ...]:
    """The default CTA size for the bin and its neighbours (half and double),
    at most one thread per pixel of the bin."""
    d = default_threads(bw * bh)
    return tuple(t for t in THREAD_CHOICES if d // 2 <= t <= 2 * d and t <= max(64, bw * bh))


def features(scene: DeviceScene) -> str:
    """Workload class of a scene: log2 buckets of pixels and triangles, the
    triangles-per-pixel density bucket, and the shading mode."""
    px = scene.width * scene.height
    T = max(1, scene.num_triangles)
    return "px%d_t%d_d%d_m%d" % (round(math.log2(px) * 2), round(math.log2(T) * 2),
                                 round(math.log2(T / px) * 2), scene.shade_mode)


class Autotuner:
    def __init__(self, bins: Iterable[Tuple[int, int]] = DEFAULT_BINS,
                 schedules: Iterable[str] = DEFAULT_SCHEDULES, reps: int = 3, cache_path: Optional[str] = None,
                 tune_threads: bool = True, other_mappings: Iterable[str] = OTHER_MAPPINGS,
                 tune_exact: bool = True):
        self.bins = tuple(tuple(b) for b in bins)
        self.tune_exact = tune_exact
        self.schedules = tuple(schedules)
        self.other_mappings = tuple(other_mappings)
        self.tune_threads = tune_threads
        self.reps = reps
        self.cache: Dict[str, dict] = {}
        self.cache_path = cache_path
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.cache = json.load(f)
        self._handles: Dict[tuple, Rasterizer] = {}

    def _handle(self, W, H, bw, bh, sched, threads=0, exact=0) -> Rasterizer:
        k = (W, H, bw, bh, sched, threads, exact)
        if k not in self._handles:
            r = Rasterizer(W, H, bw, bh, sched)
            if threads:
                r.set_option(L.PIKO_OPT_THREADS_PER_TILE, threads)
            if exact:
                r.set_option(L.PIKO_OPT_EXACT_BINS, 1)
            self._handles[k] = r
        return self._handles[k]

    def time_candidate(self, scene: DeviceScene, bw: int, bh: int, sched: str, threads: int = 0,
                       exact: int = 0) -> float:
        """Median forward time in ms of one candidate (after a sizing pass);
        threads 0 keeps the library's CTA size; exact 1 bins by the exact
        overlap test."""
        r = self._handle(scene.width, scene.height, bw, bh, sched, threads, exact)
        fb = r.forward(scene)  # sizes the bin lists
        r.status()
        times: List[float] = []
        for _ in range(self.reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            r.forward(scene, fb)
            b.record()
            b.synchronize()
            times.append(a.elapsed_time(b))
        times.sort()
        return times[len(times) // 2]

    def tune(self, scene: DeviceScene) -> dict:
        best = None
        trials = []
        for bw, bh in self.bins:
            threads = thread_candidates(bw, bh) if self.tune_threads else (default_threads(bw * bh),)
            for sched in self.schedules:
                for th in threads:
                    ms = self.time_candidate(scene, bw, bh, sched, th)
                    trials.append({"bin": [bw, bh], "schedule": sched, "threads": th, "ms": ms})
                    if best is None or ms < best["ms"]:
                        best = {"bin": [bw, bh], "schedule": sched, "threads": th, "ms": ms}
        if self.tune_exact and best is not None:
            bw, bh = best["bin"]
            ms = self.time_candidate(scene, bw, bh, best["schedule"], best["threads"], exact=1)
            trials.append({"bin": [bw, bh], "schedule": best["schedule"], "threads": best["threads"],
                           "exact_bins": 1, "ms": ms})
            if ms < best["ms"]:
                best = dict(best, exact_bins=1, ms=ms)
        bw, bh = self.bins[0] if self.bins else (16, 16)
        for sched in self.other_mappings:
            th = default_threads(bw * bh)
            ms = self.time_candidate(scene, bw, bh, sched, th)
            trials.append({"bin": [bw, bh], "schedule": sched, "threads": th, "ms": ms})
            if best is None or ms < best["ms"]:
                best = {"bin": [bw, bh], "schedule": sched, "threads": th, "ms": ms}
        best["trials"] = trials
        return best

    def knobs(self, scene: DeviceScene) -> dict:
        """The tuned bin size, schedule and threads per bin of the scene's
        workload class (measured on the first scene of the class)."""
        key = features(scene)
        if key not in self.cache:
            self.cache[key] = self.tune(scene)
        c = self.cache[key]
        bw, bh = c["bin"]
        return {"bin": (bw, bh), "schedule": c["schedule"], "threads": c.get("threads", default_threads(bw * bh)),
                "exact_bins": c.get("exact_bins", 0)}

    def choose(self, scene: DeviceScene) -> Tuple[Tuple[int, int], str]:
        k = self.knobs(scene)
        return k["bin"], k["schedule"]

    def choose_all(self, scenes: List[DeviceScene]):
        """Per-scene (bin sizes, schedules) lists for forward_batch."""
        picks = [self.choose(s) for s in scenes]
        return [p[0] for p in picks], [p[1] for p in picks]

    def _time_batch(self, r: Rasterizer, scenes: List[DeviceScene], bins, scheds, fbs=None) -> float:
        fbs = r.forward_batch(scenes, fbs, bins, scheds)  # sizes the bin lists
        r.status()
        times: List[float] = []
        for _ in range(self.reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            r.forward_batch(scenes, fbs, bins, scheds)
            b.record()
            b.synchronize()
            times.append(a.elapsed_time(b))
        times.sort()
        return times[len(times) // 2]

    def tune_batch(self, scenes: List[DeviceScene]):
        """Per-scene (bin sizes, schedules) for forward_batch, measured in the
        batched pass.  Returns (bins, schedules, report)."""
        n = len(scenes)
        cands = [((bw, bh), sc) for bw, bh in self.bins for sc in self.schedules if sc in BATCH_SCHEDULES]
        r = Rasterizer(64, 64)
        try:
            uniform = []
            for wh, sc in cands:
                uniform.append((self._time_batch(r, scenes, [wh] * n, [sc] * n), wh, sc))
            uniform.sort(key=lambda u: u[0])
            best_ms, best_wh, best_sc = uniform[0]
            classes: Dict[str, List[int]] = {}
            for i, s in enumerate(scenes):
                classes.setdefault(features(s), []).append(i)
            pick: Dict[str, Tuple[Tuple[int, int], str]] = {}
            for key, idx in classes.items():
                sub = [scenes[i] for i in idx]
                trial = [(self._time_batch(r, sub, [wh] * len(sub), [sc] * len(sub)), wh, sc) for wh, sc in cands]
                trial.sort(key=lambda u: u[0])
                pick[key] = (trial[0][1], trial[0][2])
            bins = [pick[features(s)][0] for s in scenes]
            scheds = [pick[features(s)][1] for s in scenes]
            mixed_ms = self._time_batch(r, scenes, bins, scheds)
            report = {"uniform": [{"bin": list(u[1]), "schedule": u[2], "ms": u[0]} for u in uniform],
                      "classes": len(classes), "per_class_ms": mixed_ms, "best_uniform_ms": best_ms}
            if mixed_ms < best_ms:
                report["choice"] = "per_class"
                return bins, scheds, report
            report["choice"] = "uniform"
            return [best_wh] * n, [best_sc] * n, report
        finally:
            r.close()

    def save(self, path: Optional[str] = None):
        path = path or self.cache_path
        if path:
            with open(path, "w") as f:
                json.dump(self.cache, f, indent=1, sort_keys=True)

    def close(self):
        for r in self._handles.values():
            r.close()
        self._handles.clear()
