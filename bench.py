#!/usr/bin/env python3
"""Throughput of the binned forward rasterizer on one GB300 (or N replicas).

Workload: a displaced heightfield grid of 1000 x 500 quads (1,000,000
triangles, 501,501 vertices) seen by a perspective camera at 1920 x 1080,
Lambert shading with the material and light of Listing 1, 16 x 16 tiles,
one CTA per tile (the hardware schedule; ``--schedule`` picks the static or
dynamic one).  One step = one forward pass: vertex stage, setup and
bin counts, scan, scatter, per-tile Process (coverage, depth, shading,
write-out).  Inputs are resident in HBM; the L2 is flushed between steps by
writing a 256 MiB buffer outside the per-step events.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
(the plain rasterizer the CUDA path is checked against) on bounded samples
of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mtris/s + shaded Gfrag/s on 1 GB300 (plain vs batched), bit-exact depth/ID"
UNIT = "Mtris/s"
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "process_heightfield1080p_traffic.json")
KERNEL_SOURCES = ["paper_1404_6293_gb300/csrc/piko_process.cu", "paper_1404_6293_gb300/csrc/piko_tile.cuh",
                  "paper_1404_6293_gb300/csrc/piko_internal.cuh"]

# Per-unit algorithmic costs of the Process kernel (thread operations), fixed
# before the first measurement from the minimal operation sequence of the
# definition (vertex setup per bin entry, edge tests per sample, exact depth
# and key per covered sample, shading per pixel).
OPS_PER_ENTRY = 60      # re-derive the triangle: 3 gathers, 6 differences, 64-bit area, clip to tile
OPS_PER_TEST = 12       # three 64-bit incremental edge updates and the sign test
OPS_PER_FRAGMENT = 16   # 64-bit depth numerator, reciprocal estimate and fix-up, key, shared-memory min
OPS_PER_SHADE = {0: 20, 1: 30, 2: 30}
ALU_OPS_PER_SM_CLK = 4 * 32  # four schedulers, 32 lanes


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled while the timed region runs."""

    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index: int, period_ms: int = 100):
        self.proc = None
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS), "--format=csv,noheader,nounits",
                 "-lms", str(period_ms), "-i", str(index)], stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def mark(self):
        self.out.flush()
        try:
            return sum(1 for _ in open(self.out.name))
        except OSError:
            return 0

    def stop(self, first_line: int = 0) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.flush()
        rows = [ln.strip().split(",") for ln in open(self.out.name)][first_line:]
        os.unlink(self.out.name)
        rows = [[c.strip() for c in r] for r in rows if len(r) == len(self.FIELDS)]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()), default=None)}


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The job's time is its slowest rank's: MAX all-reduce (identity on one rank)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, ms: float, scale: float = 1e6) -> float:
    """Whole-job throughput: every rank processes its own replica of the
    workload (weak scaling), so the job moves world x units in the slowest
    rank's time."""
    return world * units_per_rank / (ms * 1e-3) / scale


def workload(args):
    from paper_1404_6293_gb300 import scenes as S
    scene = S.heightfield()
    cfg = {"workload": "heightfield 1920x1080, 1000x500 quads (1,000,000 triangles), Lambert",
           "width": scene.width, "height": scene.height, "triangles": scene.num_triangles,
           "vertices": scene.num_vertices, "bin": [args.bins, args.bins], "schedule": args.schedule,
           "l2": "flushed between steps (256 MiB write outside the per-step events)"}
    return scene, cfg


def cpu_baseline(scene, seconds: float, perspective: bool = False) -> dict:
    """The oracle as it stands: bounding-box loop on all host cores + float64 shading."""
    import oracle
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    reps, t0 = 0, time.perf_counter()
    while True:
        key, _ = oracle.raster_bbox(scene, threads=cores)
        oracle.shade(scene, key, perspective=perspective)
        reps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = (time.perf_counter() - t0) / reps
    return {"value": scene.num_triangles / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{reps} full frame(s) of the same workload: bounding-box oracle on {cores} threads "
                      f"plus float64 shading, {dt:.2f} s per frame"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    from paper_1404_6293_gb300 import scenes as S
    scene, cfg = workload(args)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)

    def sub(n):
        return S.Scene(scene.width, scene.height, scene.pos, np.ascontiguousarray(scene.tris[:n]),
                       normal=scene.normal, mvp=scene.mvp, light_dir=scene.light_dir, shade_mode=scene.shade_mode)

    def step(sc):
        key, _ = oracle.raster_bbox(sc, threads=cores)
        oracle.shade(sc, key)

    # size the per-step sample so that warm-up plus timed steps stay near two minutes
    n = scene.num_triangles // 32
    t0 = time.perf_counter()
    step(sub(n))
    t1 = time.perf_counter() - t0
    budget = 120.0 / max(1, args.steps + args.warmup)
    n = int(max(2000, min(scene.num_triangles, n * budget / max(t1, 1e-6))))
    sc = sub(n)
    for _ in range(args.warmup):
        step(sc)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step(sc)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = n / (ms * 1e-3) / 1e6
    sample = (f"first {n} triangles (a contiguous band of the grid) of the workload per step, "
              f"bounding-box oracle on {cores} threads plus float64 shading")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64+f64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene, Framebuffer, Rasterizer

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    scene, cfg = workload(args)
    T = scene.num_triangles
    if args.autotune:
        # the tuner's pick of bin size, schedule and threads per bin, by forward time
        from paper_1404_6293_gb300.autotune import Autotuner
        tuner = Autotuner(reps=5)
        t0 = time.perf_counter()
        knobs = tuner.knobs(DeviceScene.from_host(scene))
        tune_s = time.perf_counter() - t0
        n_trials = len(next(iter(tuner.cache.values()))["trials"])
        tuner.close()
        args.bins, args.schedule, args.threads = knobs["bin"][0], knobs["schedule"], knobs["threads"]
        cfg.update({"bin": list(knobs["bin"]), "schedule": args.schedule,
                    "knobs": f"autotuned: fastest forward of {n_trials} candidates ({tune_s:.1f} s, untimed)"})
    r = Rasterizer(scene.width, scene.height, args.bins, args.bins, args.schedule)
    if args.threads:
        r.set_option(L.PIKO_OPT_THREADS_PER_TILE, args.threads)
        cfg["threads_per_tile"] = args.threads
    if args.perspective:
        r.set_option(L.PIKO_OPT_PERSPECTIVE, 1)
        cfg["attributes"] = "perspective-correct"
    if args.small_px:
        r.set_option(L.PIKO_OPT_SMALL_TRI_PIXELS, args.small_px)
        cfg["small_tri_pixels"] = args.small_px
    ds = DeviceScene.from_host(scene)
    fb = Framebuffer.allocate(scene.width, scene.height, scene.shade_mode)
    r.forward(ds, fb)  # sizes the bin lists (capacity check on)
    code, need = r.status()
    if code != 0:
        raise RuntimeError(f"forward status {code}")
    r.set_option(L.PIKO_OPT_CHECK_CAPACITY, 0)
    r.set_option(L.PIKO_OPT_STATS, 1)
    r.forward(ds, fb)
    stats = r.stats()
    r.set_option(L.PIKO_OPT_STATS, 0)
    covered = int((fb.key != -1).sum().item())

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    clocks = ClockSampler(torch.cuda.current_device() if world == 1 else local)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        flush.zero_()
        r.forward(ds, fb)
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for a, b in ev:
        a.record(stream)
        b.record(stream)
    barrier()
    first_clock_line = clocks.mark()
    wall0 = time.perf_counter()
    for k in range(K):
        flush.zero_()
        ev[k][0].record(stream)
        r.forward(ds, fb)
        ev[k][1].record(stream)
    barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop(first_clock_line)
    code, _ = r.status()
    if code != 0:
        raise RuntimeError(f"status {code} after the timed loop")
    step_ms = [a.elapsed_time(b) for a, b in ev]
    # per-stage times in a separate loop: events between the stages would
    # break the launch overlap the timed loop has
    Ks = min(K, 500)
    sev = [[torch.cuda.Event(enable_timing=True) for _ in range(L.PIKO_NUM_STAGE_EVENTS)] for _ in range(Ks)]
    for row in sev:
        for e in row:
            e.record(stream)
    barrier()
    for k in range(Ks):
        flush.zero_()
        r.set_stage_events(sev[k])
        r.forward(ds, fb)
    barrier()
    stage_ms = np.array([[sev[k][i].elapsed_time(sev[k][i + 1]) for i in range(L.PIKO_NUM_STAGE_EVENTS - 1)]
                         for k in range(Ks)])
    ms = max_over_ranks(float(np.sum(step_ms) / K), dist, "cuda")
    value = job_throughput(T, world, ms)
    shaded_gfrag = job_throughput(covered, world, ms, 1e9)

    # ---------------------------------------------------------------- roofline
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    proc_ms = float(stage_ms[:, 4].mean())
    V = scene.num_vertices
    attr = 12 * V * ((scene.normal is not None) + (scene.color is not None))
    bytes_proc = (4 * stats["bin_entries"] + 12 * stats["binned_triangles"] + 16 * V + attr
                  + 24 * scene.width * scene.height)
    ops_proc = (OPS_PER_ENTRY * stats["bin_entries"] + OPS_PER_TEST * stats["samples_tested"]
                + OPS_PER_FRAGMENT * stats["fragments"] + OPS_PER_SHADE[scene.shade_mode] * stats["shaded"])
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    f_mhz = (clk or {}).get("sm_mhz") or float(peaks.get("clocks_under_load", {}).get("sm_mhz_median", 1470.0))
    alu_peak = n_sm * ALU_OPS_PER_SM_CLK * f_mhz * 1e6 / 1e9  # Gop/s
    t_hbm = bytes_proc / (hbm * 1e9)
    t_alu = ops_proc / (alu_peak * 1e9)
    traffic = None
    try:
        with open(PROFILE_TRAFFIC) as f:
            prof = json.load(f)
        bin_px = args.bins * args.bins
        launch = {"bins": args.bins, "schedule": args.schedule,
                  "threads": args.threads or (64 if bin_px <= 64 else (128 if bin_px <= 256 else 256)),
                  "perspective": bool(args.perspective)}
        # counters apply only to the same kernel sources in the same launch configuration
        if prof.get("kernel_hash") == kernel_hash() and prof.get("launch") == launch:
            traffic = prof.get("dram_bytes_per_launch")
    except (OSError, ValueError):
        pass
    if t_alu >= t_hbm:
        achieved = ops_proc / (proc_ms * 1e-3) / 1e9
        roof = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Gop/s",
                "frac": achieved / alu_peak, "traffic": traffic,
                "peak_note": f"{n_sm} SMs x 128 thread-ops/clk x {f_mhz:.0f} MHz measured SM clock"}
    else:
        achieved = bytes_proc / (proc_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic, "peak_note": "of measured (MEASURED_PEAKS.json hbm_gbs)"}
    roof.update({"kernel": "k_process", "kernel_ms": proc_ms, "algorithmic_bytes": bytes_proc,
                 "algorithmic_ops": ops_proc, "t_hbm_us": t_hbm * 1e6, "t_alu_us": t_alu * 1e6,
                 "frac_at_2070mhz": (max(t_hbm, ops_proc / (n_sm * 128 * 2070e6)) / (proc_ms * 1e-3)),
                 "forward_frac": max(t_hbm, t_alu) / (ms * 1e-3)})

    # ---------------------------------------------------------------- end to end
    e2e = None
    r.set_stage_events(None)
    if not args.no_e2e:
        names = [n for n in ("pos", "tris", "normal", "color", "mvp", "light_dir") if getattr(ds, n) is not None]
        host_in = {n: getattr(ds, n).cpu().pin_memory() for n in names}
        key_h = torch.empty_like(fb.key, device="cpu").pin_memory()
        rgba_h = torch.empty_like(fb.rgba, device="cpu").pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in host_in.values())
        d2h = key_h.numel() * 8 + rgba_h.numel() * 4
        Ke = min(K, args.e2e_steps)
        pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(Ke)]
        for _ in range(3):
            r.render_from_host(host_in, ds, fb, key_h, rgba_h)
        barrier()
        # one frame at a time (L2 flushed between frames, outside the events)
        for k in range(Ke):
            flush.zero_()
            pairs[k][0].record(stream)
            r.render_from_host(host_in, ds, fb, key_h, rgba_h)
            pairs[k][1].record(stream)
        barrier()
        seq_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in pairs) / Ke, dist, "cuda")
        # frames alternate over two handles and two streams, so frame k+1's
        # host-to-device copy runs while frame k renders and copies back; every
        # frame still copies all its inputs in and its key and RGBA out
        nl = max(2, args.e2e_lanes)
        lanes = [(r, ds, fb, key_h, rgba_h)]
        for _ in range(nl - 1):
            rr = Rasterizer(scene.width, scene.height, args.bins, args.bins, args.schedule)
            if args.threads:
                rr.set_option(L.PIKO_OPT_THREADS_PER_TILE, args.threads)
            if args.perspective:
                rr.set_option(L.PIKO_OPT_PERSPECTIVE, 1)
            d = DeviceScene.from_host(scene)
            f = Framebuffer.allocate(scene.width, scene.height, scene.shade_mode)
            rr.forward(d, f)
            if rr.status()[0] != 0:
                raise RuntimeError("status error sizing an end-to-end handle")
            rr.set_option(L.PIKO_OPT_CHECK_CAPACITY, 0)
            lanes.append((rr, d, f, torch.empty_like(key_h).pin_memory(), torch.empty_like(rgba_h).pin_memory()))
        side = [torch.cuda.Stream() for _ in range(nl)]
        for k in range(3 * nl):
            rr, d, f, kh, rh = lanes[k % nl]
            rr.render_from_host(host_in, d, f, kh, rh, stream=side[k % nl])
        barrier()
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for sd in side:
            sd.wait_stream(stream)
        for k in range(Ke):
            rr, d, f, kh, rh = lanes[k % nl]
            rr.render_from_host(host_in, d, f, kh, rh, stream=side[k % nl])
        for sd in side:
            stream.wait_stream(sd)
        e1.record(stream)
        barrier()
        e_ms = max_over_ranks(e0.elapsed_time(e1) / Ke, dist, "cuda")
        # the same frames' copies alone, on the same lanes and streams: the
        # floor that the end-to-end frames cannot go below
        flush.zero_()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for sd in side:
            sd.wait_stream(stream)
        for k in range(Ke):
            rr, d, f, kh, rh = lanes[k % nl]
            with torch.cuda.stream(side[k % nl]):
                for n, t in host_in.items():
                    getattr(d, n).copy_(t, non_blocking=True)
                kh.copy_(f.key, non_blocking=True)
                rh.copy_(f.rgba, non_blocking=True)
        for sd in side:
            stream.wait_stream(sd)
        c1.record(stream)
        barrier()
        c_ms = max_over_ranks(c0.elapsed_time(c1) / Ke, dist, "cuda")
        e2e = {"value": job_throughput(T, world, e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": e_ms, "steps": Ke,
               "how": "Rasterizer.render_from_host per frame: pinned host -> device copies of every input, "
                      f"forward, device -> host copies of key and RGBA; frames rotate over {nl} handles and "
                      f"{nl} streams so copies overlap the other frames' work",
               "sequential": {"value": job_throughput(T, world, seq_ms), "ms_per_step": seq_ms,
                              "how": "one frame at a time on one stream, L2 flushed between frames"},
               "copies_only": {"ms_per_step": c_ms, "gb_s": (h2d + d2h) / (c_ms * 1e6),
                               "frac_of_e2e_time": c_ms / e_ms,
                               "how": "the same frames' host<->device copies without the forward pass"}}
        if any(ln[0].status()[0] != 0 for ln in lanes):
            raise RuntimeError("status error after the end-to-end loop")
        for ln in lanes[1:]:
            ln[0].close()

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64+f32", "data": "synthetic", "config": cfg, "shaded_gfrag_s": shaded_gfrag,
            "rasterized_gfrag_s": job_throughput(stats["fragments"], world, ms, 1e9),
            "stage_ms": {n: float(stage_ms[:, i].mean()) for i, n in
                         enumerate(["vertex", "setup_count", "scan", "scatter", "process"])},
            "work": {**stats, "covered_pixels": covered},
            "wall_ms_incl_flush": 1e3 * wall / K,
            "roofline": roof, "clocks": clk, "e2e": e2e,
            "gpu_launches": 5 * K,
            "parity": "depth/ID bit-exact vs the CPU oracle in tests/test_gpu_parity.py (same workload)"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(scene, args.cpu_seconds, args.perspective)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def _timed_steps(step, K, warmup, flush, stream):
    import torch
    for _ in range(warmup):
        flush.zero_()
        step(None)
    torch.cuda.synchronize()
    records = []
    for _ in range(K):
        flush.zero_()
        marks = {}
        step(marks)
        records.append(marks)
    torch.cuda.synchronize()
    return records


def run_extra(args):
    """Measurements of the other rows of the hot path (one GPU, rank 0):
    deferred: power-law 1080p G-buffer forward + 64-light pass;
    sphere: 64 views of a 99.5k-triangle sphere, forward + L2-loss backward."""
    import numpy as np
    import torch

    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300 import scenes as S
    from paper_1404_6293_gb300.raster import DeviceScene, Framebuffer, Rasterizer

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)  # creates the underlying CUDA event
        return e
    clocks = ClockSampler(0)
    line = {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic"}

    if args.workload == "deferred":
        scene = S.power_law_triangles()
        lights = torch.from_numpy(S.point_lights(scene.width, scene.height, 64)).cuda()
        r = Rasterizer(scene.width, scene.height, args.bins, args.bins, args.schedule)
        if args.small_px:
            r.set_option(L.PIKO_OPT_SMALL_TRI_PIXELS, args.small_px)
        if args.threads:
            r.set_option(L.PIKO_OPT_THREADS_PER_TILE, args.threads)
        ds = DeviceScene.from_host(scene)
        fb = Framebuffer.allocate(scene.width, scene.height, scene.shade_mode)
        out = torch.empty((scene.height, scene.width, 4), dtype=torch.float32, device="cuda")
        r.forward(ds, fb)
        assert r.status()[0] == 0
        r.set_option(L.PIKO_OPT_CHECK_CAPACITY, 0)
        r.set_option(L.PIKO_OPT_STATS, 1)
        r.forward(ds, fb)
        stats = r.stats()
        r.set_option(L.PIKO_OPT_STATS, 0)
        covered = int((fb.key != -1).sum().item())

        def step(m):
            if m is None:
                r.forward(ds, fb)
                r.deferred_light(fb, lights, out)
                return
            m["stage"] = [ev() for _ in range(L.PIKO_NUM_STAGE_EVENTS)]
            m["light_end"] = ev()
            r.set_stage_events(m["stage"])
            r.forward(ds, fb)
            r.deferred_light(fb, lights, out)
            m["light_end"].record(stream)

        mark = clocks.mark()
        recs = _timed_steps(step, args.steps, args.warmup, flush, stream)
        clk = clocks.stop(mark)
        assert r.status()[0] == 0
        fwd = np.array([m["stage"][0].elapsed_time(m["stage"][5]) for m in recs])
        light = np.array([m["stage"][5].elapsed_time(m["light_end"]) for m in recs])
        proc = np.array([m["stage"][4].elapsed_time(m["stage"][5]) for m in recs])
        ms = float((fwd + light).mean())
        light_ops = 30 * covered * 64
        alu_peak = n_sm * 128 * ((clk or {}).get("sm_mhz") or 1470.0) * 1e6 / 1e9
        light_bytes = scene.width * scene.height * (8 + 8 + 8 + 16)
        lt = float(light.mean()) * 1e-3
        line.update({"value": scene.num_triangles / (ms * 1e-3) / 1e6, "ms_per_step": ms, "dtype": "int64+f32",
                     "config": {"workload": "power-law 1920x1080, 500k triangles, G-buffer + 64 point lights",
                                "bin": [args.bins, args.bins], "schedule": args.schedule,
                                "l2": "flushed between steps (256 MiB write)",
                                **({"small_tri_pixels": args.small_px} if args.small_px else {}),
                                **({"threads_per_tile": args.threads} if args.threads else {})},
                     "forward_ms": float(fwd.mean()), "process_ms": float(proc.mean()),
                     "light_pass_ms": float(light.mean()),
                     "light_gpixlights_s": covered * 64 / lt / 1e9, "work": {**stats, "covered_pixels": covered},
                     "roofline": {"kernel": "k_deferred_light", "bound": "alu" if light_ops / (alu_peak * 1e9) >
                                  light_bytes / (hbm * 1e9) else "hbm",
                                  "achieved": light_ops / lt / 1e9, "peak": alu_peak, "unit": "Gop/s",
                                  "frac": light_ops / lt / 1e9 / alu_peak, "traffic": None,
                                  "hbm_frac": light_bytes / lt / 1e9 / hbm},
                     "clocks": clk, "gpu_launches": 6 * args.steps})
        if not args.no_cpu_baseline:
            import oracle
            t0 = time.perf_counter()
            key, _ = oracle.raster_bbox(scene, threads=len(os.sched_getaffinity(0)))
            gn, ga = oracle.shade(scene, key)
            oracle.light_pass(key, gn, ga, lights.cpu().numpy())
            dt = time.perf_counter() - t0
            line["cpu_baseline"] = {"value": scene.num_triangles / dt / 1e6, "unit": UNIT,
                                    "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                                    "sample": f"one full frame: bounding-box oracle, float64 G-buffer and light pass, {dt:.2f} s"}
    elif args.workload == "sphere":
        # the 64 views as one batch (scenes sharing the mesh, one camera each):
        # forward_batch, one loss-gradient op over all views, backward_batch
        # accumulating into the mesh's gradients; replayed from CUDA graphs
        import dataclasses
        sph, mvps = S.sphere_views(num_views=64)
        W = H = 512
        nv = 64
        ds = DeviceScene.from_host(sph)
        mv = torch.from_numpy(mvps).cuda()
        views = [dataclasses.replace(ds, mvp=mv[v]) for v in range(nv)]
        tgt = torch.from_numpy(S.target_image(W, H, seed=1240, views=nv)).cuda()
        key_all = torch.empty((nv, H, W), dtype=torch.int64, device="cuda")
        rgba_all = torch.empty((nv, H, W, 4), dtype=torch.float32, device="cuda")
        g_all = torch.empty_like(rgba_all)
        fbs = [Framebuffer(key_all[v], rgba_all[v]) for v in range(nv)]
        gviews = [g_all[v] for v in range(nv)]
        dc = torch.zeros_like(ds.color)
        dn = torch.zeros_like(ds.normal)
        dl = torch.zeros_like(ds.light_dir)
        bins, scheds = [(args.bins, args.bins)] * nv, ["dynamic" if args.schedule == "hardware" else args.schedule] * nv
        rb = Rasterizer(W, H, args.bins, args.bins)
        if args.perspective:
            rb.set_option(L.PIKO_OPT_PERSPECTIVE, 1)
        rb.forward_batch(views, fbs, bins, scheds)
        assert rb.status()[0] == 0
        rb.set_option(L.PIKO_OPT_CHECK_CAPACITY, 0)
        covered = int((key_all != -1).sum().item())

        def fwd_pass():
            rb.forward_batch(views, fbs, bins, scheds)

        def bwd_pass():
            dc.zero_(); dn.zero_(); dl.zero_()
            torch.sub(rgba_all, tgt, out=g_all).mul_(2.0)
            g_all[..., 3] = 0.0
            rb.backward_batch(views, fbs, gviews, [dc] * nv, [dn] * nv, [dl] * nv)

        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            for _ in range(2):
                fwd_pass(); bwd_pass()
        stream.wait_stream(side)
        torch.cuda.synchronize()
        gf, gb = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        with torch.cuda.graph(gf):
            fwd_pass()
        with torch.cuda.graph(gb):
            bwd_pass()
        torch.cuda.synchronize()

        def step(m):
            if m is not None:
                m["s"] = ev(); m["f"] = ev(); m["e"] = ev()
                m["s"].record(stream)
            gf.replay()
            if m is not None:
                m["f"].record(stream)
            gb.replay()
            if m is not None:
                m["e"].record(stream)

        mark = clocks.mark()
        recs = _timed_steps(step, args.steps, args.warmup, flush, stream)
        clk = clocks.stop(mark)
        assert rb.status()[0] == 0
        fwd = np.array([m["s"].elapsed_time(m["f"]) for m in recs])
        bwd = np.array([m["f"].elapsed_time(m["e"]) for m in recs])
        ms = float((fwd + bwd).mean())
        T = nv * sph.num_triangles
        bw_bytes = nv * W * H * (8 + 16) + sph.num_vertices * (16 + 12 * 2) + nv * sph.num_vertices * 12 * 2
        bt = float(bwd.mean()) * 1e-3
        line.update({"value": T / (ms * 1e-3) / 1e6, "ms_per_step": ms, "dtype": "int64+f32",
                     "config": {"workload": "sphere 99.5k triangles, 64 views 512x512, forward + L2 backward",
                                "bin": [args.bins, args.bins], "schedule": scheds[0],
                                "how": "the 64 views as one forward_batch and one backward_batch, each replayed "
                                       "from a CUDA graph",
                                "l2": "flushed between steps (256 MiB write)",
                                **({"attributes": "perspective-correct"} if args.perspective else {})},
                     "forward_ms": float(fwd.mean()), "backward_ms": float(bwd.mean()),
                     "covered_pixels": covered,
                     "roofline": {"kernel": "backward (64 views, incl. loss gradient)", "bound": "hbm",
                                  "achieved": bw_bytes / bt / 1e9, "peak": hbm, "unit": "GB/s",
                                  "frac": bw_bytes / bt / 1e9 / hbm, "traffic": None},
                     "clocks": clk, "gpu_launches": 2})
        if not args.no_cpu_baseline:
            import oracle
            t0 = time.perf_counter()
            sv = S.Scene(W, H, sph.pos, sph.tris, color=sph.color, normal=sph.normal, mvp=mvps[0],
                         light_dir=sph.light_dir, shade_mode=sph.shade_mode)
            key, _ = oracle.raster_bbox(sv, threads=len(os.sched_getaffinity(0)))
            rgba = oracle.shade(sv, key, perspective=args.perspective)
            gg = np.zeros((H, W, 4))
            gg[..., :3] = 2 * (rgba[..., :3] - tgt[0].cpu().numpy()[..., :3])
            oracle.backward(sv, key, gg, perspective=args.perspective)
            dt = time.perf_counter() - t0
            line["cpu_baseline"] = {"value": sph.num_triangles / dt / 1e6, "unit": UNIT,
                                    "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                                    "sample": f"one view: bounding-box oracle, float64 shading and gradients, {dt:.2f} s"}
    elif args.workload == "batch":
        line.update(run_batch(args, clocks))
    else:
        raise SystemExit(f"unknown workload {args.workload}")
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args, clocks) -> dict:
    """256 scenes (1k-200k triangles, 256^2-1024^2): plain per-scene loop of
    forward + backward (16x16 bins, static) against the autotuned batch,
    forward_batch + backward_batch replayed from one CUDA graph."""
    import numpy as np
    import torch

    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300 import scenes as S
    from paper_1404_6293_gb300.autotune import Autotuner
    from paper_1404_6293_gb300.raster import DeviceScene, Framebuffer, Rasterizer

    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    host = S.scene_batch(args.batch_scenes)
    ds = [DeviceScene.from_host(s) for s in host]
    n = len(ds)
    npx = [s.width * s.height for s in host]
    po = np.concatenate([[0], np.cumsum(npx)])
    vo = np.concatenate([[0], np.cumsum([s.num_vertices for s in host])])
    P, VT = int(po[-1]), int(vo[-1])
    T = int(sum(s.num_triangles for s in host))

    def make_fbs():
        key = torch.empty(P, dtype=torch.int64, device="cuda")
        rgba = torch.empty((P, 4), dtype=torch.float32, device="cuda")
        fbs = [Framebuffer(key[po[i]:po[i + 1]].view(host[i].height, host[i].width),
                           rgba[po[i]:po[i + 1]].view(host[i].height, host[i].width, 4)) for i in range(n)]
        return key, rgba, fbs

    def make_grads():
        dc = torch.zeros((VT, 3), device="cuda")
        dn = torch.zeros((VT, 3), device="cuda")
        dl = torch.zeros((n, 3), device="cuda")
        return dc, dn, dl, [dc[vo[i]:vo[i + 1]] for i in range(n)], [dn[vo[i]:vo[i + 1]] for i in range(n)], \
            [dl[i] for i in range(n)]

    gen = torch.Generator(device="cuda").manual_seed(1240)
    target = torch.rand((P, 4), generator=gen, device="cuda")
    g_all = torch.empty((P, 4), device="cuda")
    gviews = [g_all[po[i]:po[i + 1]].view(host[i].height, host[i].width, 4) for i in range(n)]

    # ---- plain: one handle per resolution, 16x16 bins, static
    handles = {}
    for s in host:
        if (s.width, s.height) not in handles:
            handles[(s.width, s.height)] = Rasterizer(s.width, s.height, 16, 16, "static")
    key_p, rgba_p, fbs_p = make_fbs()
    dc_p, dn_p, dl_p, dcv_p, dnv_p, dlv_p = make_grads()
    for i in range(n):
        handles[(host[i].width, host[i].height)].forward(ds[i], fbs_p[i])
    for h in handles.values():
        assert h.status()[0] == 0
        h.set_option(L.PIKO_OPT_CHECK_CAPACITY, 0)

    def plain_step():
        dc_p.zero_(); dn_p.zero_(); dl_p.zero_()
        for i in range(n):
            handles[(host[i].width, host[i].height)].forward(ds[i], fbs_p[i])
        torch.sub(rgba_p, target, out=g_all).mul_(2.0)
        g_all[:, 3] = 0.0
        for i in range(n):
            handles[(host[i].width, host[i].height)].backward(ds[i], fbs_p[i], gviews[i], dcv_p[i], dnv_p[i], dlv_p[i])

    # ---- batched: autotuned knobs, one persistent launch per pass, graph-captured
    t0 = time.perf_counter()
    if args.batch_bins:
        bins, scheds = [(args.batch_bins, args.batch_bins)] * n, [args.batch_schedule] * n
        tune_report = {"choice": "given", "classes": 0, "per_class_ms": None, "best_uniform_ms": None, "uniform": []}
    else:
        tuner = Autotuner()
        bins, scheds, tune_report = tuner.tune_batch(ds)
        tuner.close()
    tune_s = time.perf_counter() - t0
    rb = Rasterizer(64, 64, 16, 16)
    rb.set_option(L.PIKO_OPT_BATCH_LAUNCH, 1 if args.batch_launch == "per-phase" else 0)
    key_b, rgba_b, fbs_b = make_fbs()
    dc_b, dn_b, dl_b, dcv_b, dnv_b, dlv_b = make_grads()
    rb.forward_batch(ds, fbs_b, bins, scheds)
    assert rb.status()[0] == 0
    rb.set_option(L.PIKO_OPT_CHECK_CAPACITY, 0)

    def batched_step():
        dc_b.zero_(); dn_b.zero_(); dl_b.zero_()
        rb.forward_batch(ds, fbs_b, bins, scheds)
        torch.sub(rgba_b, target, out=g_all).mul_(2.0)
        g_all[:, 3] = 0.0
        rb.backward_batch(ds, fbs_b, gviews, dcv_b, dnv_b, dlv_b)

    for _ in range(2):
        batched_step()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batched_step()
    torch.cuda.synchronize()

    def timed(fn, K, W):
        for _ in range(W):
            flush.zero_()
            fn()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(K):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            tot += a.elapsed_time(b)
        return tot / K

    mark = clocks.mark()
    ms_plain = timed(plain_step, args.steps, args.warmup)
    ms_batch = timed(graph.replay, args.steps, args.warmup)
    clk = clocks.stop(mark)
    assert rb.status()[0] == 0
    same_keys = bool(torch.equal(key_p, key_b))
    gdiff = max(float((dc_p - dc_b).abs().max()), float((dn_p - dn_b).abs().max()), float((dl_p - dl_b).abs().max()))
    gscale = max(float(dc_p.abs().max()), float(dn_p.abs().max()), float(dl_p.abs().max()))
    n_static = sum(1 for x in scheds if x == "static")
    return {"value": T / (ms_batch * 1e-3) / 1e6, "ms_per_step": ms_batch, "dtype": "int64+f32",
            "config": {"workload": f"{n} scenes, 1k-200k triangles, 256^2-1024^2, random + heightfield, "
                                   "forward + L2 backward", "scenes": n, "triangles": T, "pixels": P,
                       "l2": "flushed between steps (256 MiB write)"},
            "plain": {"value": T / (ms_plain * 1e-3) / 1e6, "ms_per_step": ms_plain,
                      "how": "per-scene piko_raster_forward then piko_raster_backward, 16x16 static"},
            "batched": {"value": T / (ms_batch * 1e-3) / 1e6, "ms_per_step": ms_batch,
                        "how": ("forward_batch (one persistent cooperative launch)" if args.batch_launch == "persistent"
                                else "forward_batch (one launch per phase)") + " + loss gradient + "
                               "backward_batch, replayed from one CUDA graph",
                        "autotune_s": tune_s, "static_scenes": n_static,
                        "bins_used": sorted(set(f"{a}x{b}" for a, b in bins)),
                        "autotune": {"choice": tune_report["choice"], "classes": tune_report["classes"],
                                     "per_class_forward_ms": tune_report["per_class_ms"],
                                     "best_uniform_forward_ms": tune_report["best_uniform_ms"],
                                     "uniform_forward_ms": {f"{u['bin'][0]}x{u['bin'][1]} {u['schedule']}": u["ms"]
                                                            for u in tune_report["uniform"]}}},
            "speedup_batched_over_plain": ms_plain / ms_batch,
            "parity": {"keys_bit_identical_plain_vs_batched": same_keys, "grad_max_abs_diff": gdiff,
                       "grad_scale": gscale},
            "clocks": clk, "gpu_launches": (2 if args.batch_launch == "persistent" else 6) * args.steps,
            "gpu_launches_plain": 7 * n * args.steps}


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--bins", type=int, default=16)
    ap.add_argument("--schedule", default="hardware", choices=["static", "dynamic", "hardware"],
                    help="tile schedule of the heightfield line (hardware: one CTA per tile, the fastest "
                         "of the bin-size x schedule sweep at 16x16)")
    ap.add_argument("--threads", type=int, default=0, help="Process CTA size (0: library default)")
    ap.add_argument("--perspective", action="store_true",
                    help="heightfield and sphere workloads: perspective-correct attributes (PIKO_OPT_PERSPECTIVE)")
    ap.add_argument("--autotune", action="store_true",
                    help="heightfield workload: bin size, schedule and threads per bin from the autotuner")
    ap.add_argument("--small-px", type=int, default=0,
                    help="largest box (pixels inside a tile) one thread rasterizes; larger boxes take a warp "
                         "(0: library default)")
    ap.add_argument("--batch-scenes", type=int, default=256)
    ap.add_argument("--batch-bins", type=int, default=0, help="batch workload: one square bin size for all scenes "
                    "instead of the autotuner's choice (0: autotune)")
    ap.add_argument("--batch-schedule", default="dynamic", choices=["static", "dynamic"])
    ap.add_argument("--batch-launch", default="persistent", choices=["persistent", "per-phase"],
                    help="batch workload: one cooperative launch, or one launch per phase (for launch lists)")
    ap.add_argument("--workload", default="heightfield", choices=["heightfield", "deferred", "sphere", "batch"],
                    help="heightfield: the headline line; the others measure further rows of the path")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-lanes", type=int, default=3, help="handles/streams the end-to-end frames rotate over")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        sys.exit(run_reference(args))
    sys.exit(run_ours(args) if args.workload == "heightfield" else run_extra(args))


if __name__ == "__main__":
    main()
