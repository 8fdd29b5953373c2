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


_NVML_SAMPLER = r"""
import ctypes as C, sys, time
index, bus, period, out = int(sys.argv[1]), sys.argv[2], float(sys.argv[3]), sys.argv[4]
lib = C.CDLL("libnvidia-ml.so.1")
if lib.nvmlInit_v2() != 0:
    sys.exit(3)
dev = C.c_void_p()
if not (bus and lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), C.byref(dev)) == 0):
    if lib.nvmlDeviceGetHandleByIndex_v2(C.c_uint(index), C.byref(dev)) != 0:
        sys.exit(4)
reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or lib.nvmlDeviceGetCurrentClocksThrottleReasons
mx = C.c_uint(0)
mxv = mx.value if lib.nvmlDeviceGetMaxClockInfo(dev, 1, C.byref(mx)) == 0 else 0
mhz, mw, rs = C.c_uint(0), C.c_uint(0), C.c_ulonglong(0)
with open(out, "w", buffering=1) as f:
    f.write("max,%d\n" % mxv)
    while True:
        sm = mhz.value if lib.nvmlDeviceGetClockInfo(dev, 1, C.byref(mhz)) == 0 else 0
        pw = mw.value if lib.nvmlDeviceGetPowerUsage(dev, C.byref(mw)) == 0 else 0
        r = rs.value if reasons_fn(dev, C.byref(rs)) == 0 else 0
        f.write("%.6f,%d,%d,%d\n" % (time.monotonic(), sm, pw, r))
        time.sleep(period)
"""


class ClockSampler:
    """SM clock, power and clock-event reasons sampled during the timed
    regions.  A child process polls NVML (read-only queries through ctypes;
    libnvidia-ml ships with the driver) every ``period_ms`` and stamps each
    sample with the system monotonic clock, so that even a timed loop of a
    few milliseconds gets samples and the sampling takes no time from this
    process; nvidia-smi (100 ms) is the fallback when NVML cannot be loaded.
    ``mark()`` returns a time; ``summary(a, b)`` summarises the samples taken
    between two marks."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, index: int, period_ms: float = 0.5):
        self.source = "nvml"
        self._smi = None
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.out.close()
        bus = ""
        try:
            import torch
            p = torch.cuda.get_device_properties(index)
            bus = "%08X:%02X:%02X.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
        except Exception:
            bus = ""
        self.proc = subprocess.Popen([sys.executable, "-c", _NVML_SAMPLER, str(index), bus, str(period_ms * 1e-3),
                                      self.out.name], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        # wait for the first sample (or for the child to give up)
        t0 = time.monotonic()
        while time.monotonic() - t0 < 10.0:
            if self.proc.poll() is not None or len(self._rows()[1]) > 0:
                break
            time.sleep(0.01)
        if not self._rows()[1]:
            self._kill()
            self.source = "nvidia-smi"
            self._smi = _SmiSampler(index)

    def _rows(self):
        mx, rows = None, []
        try:
            for ln in open(self.out.name):
                parts = ln.strip().split(",")
                if parts[0] == "max" and len(parts) == 2:
                    mx = float(parts[1]) or None
                elif len(parts) == 4:
                    rows.append((float(parts[0]), float(parts[1]), float(parts[2]) / 1000.0, int(parts[3])))
        except (OSError, ValueError):
            pass
        return mx, rows

    def mark(self):
        if self._smi is not None:
            return self._smi.mark()
        return time.monotonic()

    def summary(self, begin, end=None) -> dict:
        if self._smi is not None:
            return self._smi.summary(begin, end)
        mx, rows = self._rows()
        rows = [r for r in rows if r[0] >= begin and (end is None or r[0] <= end)]
        sm = [r[1] for r in rows if r[1] > 0]
        pw = [r[2] for r in rows if r[2] > 0]
        reasons = sorted({name for r in rows for bit, name in self.REASONS.items() if r[3] & bit})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "sm_mhz_min": min(sm) if sm else None, "reasons": reasons, "samples": len(rows),
                "power_w_max": max(pw) if pw else None, "source": self.source}

    def stop(self, first_line=0) -> dict:
        out = self.summary(first_line)
        self.close()
        return out

    def _kill(self):
        if self.proc is not None and self.proc.poll() is None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def close(self):
        self._kill()
        if self._smi is not None:
            self._smi.close()
        try:
            os.unlink(self.out.name)
        except OSError:
            pass


class _SmiSampler:
    """nvidia-smi clocks and throttle reasons every 100 ms (fallback)."""

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

    def _rows(self):
        self.out.flush()
        try:
            rows = [ln.strip().split(",") for ln in open(self.out.name)]
        except OSError:
            return []
        return [[c.strip() for c in r] for r in rows if len(r) == len(self.FIELDS)]

    def mark(self):
        return len(self._rows())

    def summary(self, begin, end=None) -> dict:
        rows = self._rows()[begin:end]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "source": "nvidia-smi"}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows), "source": "nvidia-smi",
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()), default=None)}

    def close(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        try:
            os.unlink(self.out.name)
        except OSError:
            pass


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
           "vertices": scene.num_vertices, "bin": [args.bins, args.bin_h or args.bins], "schedule": args.schedule,
           "l2": "flushed between steps (256 MiB write outside the per-step events)"}
    return scene, cfg


# ---------------------------------------------------------------- CPU side
def host_cpu() -> dict:
    """Host cores this process may use and the CPU model (lscpu, else /proc/cpuinfo)."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.TimeoutExpired):
        pass
    if not model:
        try:
            info = open("/proc/cpuinfo").read().splitlines()
            for ln in info:
                if ln.lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
            if not model:
                impl = next((ln.split(":")[1].strip() for ln in info if ln.startswith("CPU implementer")), "?")
                part = next((ln.split(":")[1].strip() for ln in info if ln.startswith("CPU part")), "?")
                model = f"CPU implementer {impl}, part {part}"
        except OSError:
            model = "unknown"
    return {"cores": cores, "cpu_model": model}


def _repeat(fn, seconds: float):
    """Runs fn() until ``seconds`` have passed (at least once): (reps, seconds per rep)."""
    reps, t0 = 0, time.perf_counter()
    while True:
        fn()
        reps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    return reps, (time.perf_counter() - t0) / reps


def _band(scene, n):
    """The scene with only its first n triangles (same vertices, camera and shading)."""
    import dataclasses

    import numpy as np
    return dataclasses.replace(scene, tris=np.ascontiguousarray(scene.tris[:n]))


def oracle_frame_fn(scene, threads, perspective=False, extra=None):
    import oracle

    def fn():
        key, _ = oracle.raster_bbox(scene, threads=threads)
        out = oracle.shade(scene, key, perspective=perspective)
        if extra is not None:
            extra(key, out)
    return fn


def cpu_baseline(scene, seconds: float, perspective: bool = False, single_seconds: float = 3.0,
                 extra=None, what: str = "bounding-box oracle plus float64 shading") -> dict:
    """The oracle as it stands, on the host cores: full frames on every core
    (row bands), and a band of the triangles on one thread."""
    hc = host_cpu()
    cores = hc["cores"]
    reps, dt = _repeat(oracle_frame_fn(scene, cores, perspective, extra), seconds)
    T = scene.num_triangles
    # single thread: a leading band of the triangles, sized from a probe
    n = max(1, T // 64)
    t0 = time.perf_counter()
    oracle_frame_fn(_band(scene, n), 1, perspective, extra)()
    t1 = max(time.perf_counter() - t0, 1e-6)
    n = int(max(1, min(T, n * single_seconds / t1)))
    r1, d1 = _repeat(oracle_frame_fn(_band(scene, n), 1, perspective, extra), single_seconds)
    return {"value": T / dt / 1e6, "unit": UNIT, "cores": cores, "cpu_model": hc["cpu_model"], "kind": "oracle",
            "sample": f"{reps} full frame(s): {what} on {cores} threads, {dt:.3f} s per frame",
            "single_thread": {"value": n / d1 / 1e6, "unit": UNIT, "cores": 1,
                              "sample": f"first {n} of {T} triangles per frame, {r1} frame(s), {what} on one "
                                        f"thread, {d1:.3f} s per frame"}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    scene, cfg = workload(args)
    cores = host_cpu()["cores"]

    def step(sc):
        key, _ = oracle.raster_bbox(sc, threads=cores)
        oracle.shade(sc, key)

    # size the per-step sample so that warm-up plus timed steps stay near two minutes
    n = scene.num_triangles // 32
    t0 = time.perf_counter()
    step(_band(scene, n))
    t1 = time.perf_counter() - t0
    budget = 120.0 / max(1, args.steps + args.warmup)
    n = int(max(2000, min(scene.num_triangles, n * budget / max(t1, 1e-6))))
    sc = _band(scene, n)
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


# ---------------------------------------------------------------- GPU side
class Ctx:
    """What every measurement shares: stream, L2 flush buffer, peaks, clocks."""

    def __init__(self, clocks):
        import torch
        self.torch = torch
        self.stream = torch.cuda.current_stream()
        self.flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        self.peaks = measured_peaks()
        self.hbm = float(self.peaks.get("hbm_gbs", 6800.0))
        self.n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        self.clocks = clocks

    def event(self):
        e = self.torch.cuda.Event(enable_timing=True)
        e.record(self.stream)  # creates the underlying CUDA event
        return e

    def f_mhz(self, clk) -> float:
        return (clk or {}).get("sm_mhz") or float(self.peaks.get("clocks_under_load", {}).get("sm_mhz_median", 1470.0))

    def alu_peak(self, clk) -> float:
        """Thread-ops/s of the SMs at the sampled clock, in Gop/s."""
        return self.n_sm * ALU_OPS_PER_SM_CLK * self.f_mhz(clk) * 1e6 / 1e9


def time_forward(ctx, r, ds, fb, K, W, stages=True):
    """Per-step forward times (ms, CUDA events around each step on the
    launching stream, L2 flushed between steps) and, in a second loop, the
    per-stage times from the library's stage events."""
    import numpy as np
    torch = ctx.torch
    for _ in range(W):
        ctx.flush.zero_()
        r.forward(ds, fb)
    ev = [(ctx.event(), ctx.event()) for _ in range(K)]
    torch.cuda.synchronize()
    for k in range(K):
        ctx.flush.zero_()
        ev[k][0].record(ctx.stream)
        r.forward(ds, fb)
        ev[k][1].record(ctx.stream)
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    stage_ms = None
    if stages:
        from paper_1404_6293_gb300 import _lib as L
        sev = [[ctx.event() for _ in range(L.PIKO_NUM_STAGE_EVENTS)] for _ in range(K)]
        torch.cuda.synchronize()
        for k in range(K):
            ctx.flush.zero_()
            r.set_stage_events(sev[k])
            r.forward(ds, fb)
        torch.cuda.synchronize()
        r.set_stage_events(None)
        stage_ms = np.array([[sev[k][i].elapsed_time(sev[k][i + 1]) for i in range(L.PIKO_NUM_STAGE_EVENTS - 1)]
                             for k in range(K)])
    return step_ms, stage_ms


def forward_launches(W: int, H: int, bw: int, bh: int) -> int:
    """The library's kernels per single-scene forward without stage events:
    vertex, count, scan, scatter, Process; a frame of at most 2,048 bins is
    scanned by the count pass itself (one launch fewer)."""
    nbins = ((W + bw - 1) // bw) * ((H + bh - 1) // bh)
    return 4 if nbins <= 2048 else 5


def exact_bins_record(ctx, scene, ds, bins, schedule, K, W, threads=0, bin_h=0) -> dict:
    """The same forward with AssignBin's exact overlap test on (a handle of
    its own): per-step and per-stage times and bin entries, beside the
    bounding-box binning of the line."""
    import numpy as np
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import Framebuffer, Rasterizer
    rec = {}
    for exact in (0, 1):
        r = Rasterizer(scene.width, scene.height, bins, bin_h or bins, schedule)
        if threads:
            r.set_option(L.PIKO_OPT_THREADS_PER_TILE, threads)
        r.set_option(L.PIKO_OPT_EXACT_BINS, exact)
        fb = Framebuffer.allocate(scene.width, scene.height, scene.shade_mode)
        stats, _ = size_and_count(r, ds, fb)
        step_ms, stage_ms = time_forward(ctx, r, ds, fb, K, W)
        if r.status()[0] != 0:
            raise RuntimeError("status error in the exact-bins loop")
        sm = stage_ms.mean(axis=0)
        rec["exact" if exact else "bounding_box"] = {
            "forward_ms": float(np.median(step_ms)), "bin_entries": stats["bin_entries"],
            "stage_ms": dict(zip(["vertex", "setup_count", "scan", "scatter", "process"], (float(x) for x in sm)))}
        r.close()
    rec["how"] = ("PIKO_OPT_EXACT_BINS: entries only in bins the triangle overlaps (separating-axis test of its "
                  "edges against the bin's pixel centres), against bounding-box bins; same keys")
    return rec


def size_and_count(r, ds, fb):
    """One forward that sizes the bin lists, then one with the work counters:
    (stats, covered pixels).  Leaves the capacity check off and the counters off."""
    from paper_1404_6293_gb300 import _lib as L
    r.forward(ds, fb)
    code, _ = r.status()
    if code != 0:
        raise RuntimeError(f"forward status {code}")
    r.set_option(L.PIKO_OPT_CHECK_CAPACITY, 0)
    r.set_option(L.PIKO_OPT_STATS, 1)
    r.forward(ds, fb)
    stats = r.stats()
    r.set_option(L.PIKO_OPT_STATS, 0)
    return stats, int((fb.key != -1).sum().item())


def process_roofline(ctx, scene, stats, proc_ms, clk, traffic=None) -> dict:
    """Roofline of the Process kernel: algorithmic bytes (4 B per bin entry,
    12 B of indices per binned triangle, 16 B per snapped vertex, 12 B per
    vertex per attribute array, 24 B per pixel written) at the measured HBM
    copy bandwidth, against algorithmic thread-ops at the sampled SM clock."""
    V = scene.num_vertices
    attr = 12 * V * ((scene.normal is not None) + (scene.color is not None))
    bytes_proc = (4 * stats["bin_entries"] + 12 * stats["binned_triangles"] + 16 * V + attr
                  + 24 * scene.width * scene.height)
    ops_proc = (OPS_PER_ENTRY * stats["bin_entries"] + OPS_PER_TEST * stats["samples_tested"]
                + OPS_PER_FRAGMENT * stats["fragments"] + OPS_PER_SHADE[scene.shade_mode] * stats["shaded"])
    alu_peak = ctx.alu_peak(clk)
    t_hbm = bytes_proc / (ctx.hbm * 1e9)
    t_alu = ops_proc / (alu_peak * 1e9)
    if t_alu >= t_hbm:
        achieved = ops_proc / (proc_ms * 1e-3) / 1e9
        roof = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Gop/s",
                "frac": achieved / alu_peak, "traffic": traffic,
                "peak_note": f"{ctx.n_sm} SMs x 128 thread-ops/clk x {ctx.f_mhz(clk):.0f} MHz sampled SM clock"}
    else:
        achieved = bytes_proc / (proc_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": ctx.hbm, "unit": "GB/s", "frac": achieved / ctx.hbm,
                "traffic": traffic, "peak_note": "of measured (MEASURED_PEAKS.json hbm_gbs)"}
    roof.update({"kernel": "k_process", "kernel_ms": proc_ms, "algorithmic_bytes": bytes_proc,
                 "algorithmic_ops": ops_proc, "t_hbm_us": t_hbm * 1e6, "t_alu_us": t_alu * 1e6,
                 "sm_mhz_used": ctx.f_mhz(clk),
                 "frac_at_2070mhz": max(t_hbm, ops_proc / (ctx.n_sm * 128 * 2070e6)) / (proc_ms * 1e-3)})
    return roof


def headline_traffic(args):
    """ncu DRAM bytes per Process launch, when the committed record matches
    these kernel sources and this launch configuration."""
    try:
        with open(PROFILE_TRAFFIC) as f:
            prof = json.load(f)
        if args.bin_h and args.bin_h != args.bins:
            return None  # the record is for square bins
        bin_px = args.bins * args.bins
        launch = {"bins": args.bins, "schedule": args.schedule,
                  "threads": args.threads or (64 if bin_px <= 64 else (128 if bin_px <= 256 else 256)),
                  "perspective": bool(args.perspective)}
        if prof.get("kernel_hash") == kernel_hash() and prof.get("launch") == launch:
            return prof.get("dram_bytes_per_launch")
    except (OSError, ValueError):
        pass
    return None


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
        args.bin_h = knobs["bin"][1]
        args.exact_bins = knobs["exact_bins"]
        cfg.update({"bin": list(knobs["bin"]), "schedule": args.schedule,
                    "knobs": f"autotuned: fastest forward of {n_trials} candidates ({tune_s:.1f} s, untimed)"})
    r = Rasterizer(scene.width, scene.height, args.bins, args.bin_h or args.bins, args.schedule)
    if args.threads:
        r.set_option(L.PIKO_OPT_THREADS_PER_TILE, args.threads)
        cfg["threads_per_tile"] = args.threads
    if args.perspective:
        r.set_option(L.PIKO_OPT_PERSPECTIVE, 1)
        cfg["attributes"] = "perspective-correct"
    if args.small_px:
        r.set_option(L.PIKO_OPT_SMALL_TRI_PIXELS, args.small_px)
        cfg["small_tri_pixels"] = args.small_px
    if args.exact_bins:
        r.set_option(L.PIKO_OPT_EXACT_BINS, 1)
        cfg["exact_bins"] = 1
    ds = DeviceScene.from_host(scene)
    fb = Framebuffer.allocate(scene.width, scene.height, scene.shade_mode)
    stats, covered = size_and_count(r, ds, fb)

    clocks = ClockSampler(torch.cuda.current_device())
    ctx = Ctx(clocks)
    stream = ctx.stream
    for _ in range(args.warmup):
        ctx.flush.zero_()
        r.forward(ds, fb)
    K = args.steps
    ev = [(ctx.event(), ctx.event()) for _ in range(K)]
    barrier()
    mark0 = clocks.mark()
    wall0 = time.perf_counter()
    for k in range(K):
        ctx.flush.zero_()
        ev[k][0].record(stream)
        r.forward(ds, fb)
        ev[k][1].record(stream)
    barrier()
    wall = time.perf_counter() - wall0
    mark1 = clocks.mark()
    code, _ = r.status()
    if code != 0:
        raise RuntimeError(f"status {code} after the timed loop")
    step_ms = [a.elapsed_time(b) for a, b in ev]
    # per-stage times in a separate loop: events between the stages would
    # break the launch overlap the timed loop has
    _, stage_ms = time_forward(ctx, r, ds, fb, min(K, 500), 1)
    barrier()
    mark2 = clocks.mark()
    clk = clocks.summary(mark0, mark1)
    clk_both = clocks.summary(mark0, mark2)  # the timed loop and the per-stage loop: same kernels
    if not clk.get("sm_mhz"):
        clk = dict(clk_both, note="no sample inside the timed loop alone; summary over the timed and stage loops")
    clk["with_stage_loop"] = {k: clk_both.get(k) for k in ("sm_mhz", "samples", "reasons")}
    ms = max_over_ranks(float(np.sum(step_ms) / K), dist, "cuda")
    value = job_throughput(T, world, ms)
    shaded_gfrag = job_throughput(covered, world, ms, 1e9)
    proc_ms = float(stage_ms[:, 4].mean())
    roof = process_roofline(ctx, scene, stats, proc_ms, clk, headline_traffic(args))
    roof["forward_frac"] = max(roof["t_hbm_us"], roof["t_alu_us"]) * 1e-3 / ms

    e2e = None if args.no_e2e else measure_e2e(args, ctx, r, ds, fb, scene, world, dist, barrier)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64+f32", "data": "synthetic", "config": cfg, "shaded_gfrag_s": shaded_gfrag,
            "rasterized_gfrag_s": job_throughput(stats["fragments"], world, ms, 1e9),
            "stage_ms": {n: float(stage_ms[:, i].mean()) for i, n in
                         enumerate(["vertex", "setup_count", "scan", "scatter", "process"])},
            "work": {**stats, "covered_pixels": covered},
            "wall_ms_incl_flush": 1e3 * wall / K,
            "step_ms_min": float(np.min(step_ms)), "step_ms_median": float(np.median(step_ms)),
            "roofline": roof, "clocks": clk, "e2e": e2e,
            "gpu_launches": forward_launches(scene.width, scene.height, args.bins, args.bin_h or args.bins) * K,
            "parity": "depth/ID bit-exact vs the CPU oracle on this workload under every schedule "
                      "(tests/test_gpu_full_size.py)"}
    if rank == 0 and world == 1 and not args.no_configs:
        line["bin_sweep"] = bin_sweep(args, ctx, scene, ds)
        line["exact_bins"] = exact_bins_record(ctx, scene, ds, args.bins, args.schedule, K, args.warmup,
                                               args.threads, args.bin_h)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(scene, args.cpu_seconds, args.perspective)
    if rank == 0 and world == 1 and not args.no_configs:
        line["configs"] = {
            "C1_random_256": measure_random256(args, ctx),
            "C3_deferred_powerlaw_1080p": measure_deferred(args, ctx),
            "C4_sphere_64_views": measure_sphere(args, ctx),
            "C5_batch_256_scenes": measure_batch(args, ctx),
            "F4_reyes_sample": measure_reyes(args, ctx),
        }
    clocks.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def measure_e2e(args, ctx, r, ds, fb, scene, world, dist, barrier) -> dict:
    """The same metric through the C ABI with host buffers
    (piko_raster_forward_host via Rasterizer.forward_host): every frame the
    library copies the scene's pinned host arrays to the device, runs the
    forward pass and copies key and RGBA into pinned host arrays, all inside
    the events."""
    import torch

    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene, Framebuffer, HostScene, Rasterizer
    T = scene.num_triangles
    stream = ctx.stream
    K = args.steps
    hs = HostScene.from_host(scene)  # pinned; read-only, shared by every lane
    names = [n for n in ("pos", "tris", "normal", "color", "mvp", "light_dir") if getattr(hs, n) is not None]
    host_in = {n: getattr(hs, n) for n in names}

    def host_fb():
        return Framebuffer(torch.empty_like(fb.key, device="cpu").pin_memory(),
                           torch.empty_like(fb.rgba, device="cpu").pin_memory())

    fb_h = host_fb()
    h2d = sum(t.numel() * t.element_size() for t in host_in.values())
    d2h = fb_h.key.numel() * 8 + fb_h.rgba.numel() * 4
    Ke = min(K, args.e2e_steps)
    pairs = [(ctx.event(), ctx.event()) for _ in range(Ke)]
    for _ in range(3):
        r.forward_host(hs, fb_h, stream)
    barrier()
    # one frame at a time (L2 flushed between frames, outside the events)
    for k in range(Ke):
        ctx.flush.zero_()
        pairs[k][0].record(stream)
        r.forward_host(hs, fb_h, stream)
        pairs[k][1].record(stream)
    barrier()
    seq_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in pairs) / Ke, dist, "cuda")
    # frames rotate over several handles and streams, so frame k+1's
    # host-to-device copy runs while frame k renders and copies back; every
    # frame still copies all its inputs in and its key and RGBA out
    nl = max(2, args.e2e_lanes)
    lanes = [(r, fb_h, ds, fb)]
    for _ in range(nl - 1):
        rr = Rasterizer(scene.width, scene.height, args.bins, args.bin_h or args.bins, args.schedule)
        if args.threads:
            rr.set_option(L.PIKO_OPT_THREADS_PER_TILE, args.threads)
        if args.perspective:
            rr.set_option(L.PIKO_OPT_PERSPECTIVE, 1)
        if args.small_px:
            rr.set_option(L.PIKO_OPT_SMALL_TRI_PIXELS, args.small_px)
        f_h = host_fb()
        rr.forward_host(hs, f_h, stream)
        torch.cuda.synchronize()
        if rr.status()[0] != 0:
            raise RuntimeError("status error sizing an end-to-end handle")
        rr.set_option(L.PIKO_OPT_CHECK_CAPACITY, 0)
        # device tensors of the same shapes for the copies-only leg below
        lanes.append((rr, f_h, DeviceScene.from_host(scene), Framebuffer.allocate(scene.width, scene.height,
                                                                                   scene.shade_mode)))
    side = [torch.cuda.Stream() for _ in range(nl)]
    for k in range(3 * nl):
        rr, f_h = lanes[k % nl][:2]
        rr.forward_host(hs, f_h, side[k % nl])
    barrier()
    ctx.flush.zero_()
    e0, e1 = ctx.event(), ctx.event()
    e0.record(stream)
    for sd in side:
        sd.wait_stream(stream)
    for k in range(Ke):
        rr, f_h = lanes[k % nl][:2]
        rr.forward_host(hs, f_h, side[k % nl])
    for sd in side:
        stream.wait_stream(sd)
    e1.record(stream)
    barrier()
    e_ms = max_over_ranks(e0.elapsed_time(e1) / Ke, dist, "cuda")
    # the same frames' copies alone, on the same lanes and streams: the
    # floor that the end-to-end frames cannot go below
    ctx.flush.zero_()
    c0, c1 = ctx.event(), ctx.event()
    c0.record(stream)
    for sd in side:
        sd.wait_stream(stream)
    for k in range(Ke):
        _, f_h, d, f = lanes[k % nl]
        with torch.cuda.stream(side[k % nl]):
            for n, t in host_in.items():
                getattr(d, n).copy_(t, non_blocking=True)
            f_h.key.copy_(f.key, non_blocking=True)
            f_h.rgba.copy_(f.rgba, non_blocking=True)
    for sd in side:
        stream.wait_stream(sd)
    c1.record(stream)
    barrier()
    c_ms = max_over_ranks(c0.elapsed_time(c1) / Ke, dist, "cuda")
    if any(ln[0].status()[0] != 0 for ln in lanes):
        raise RuntimeError("status error after the end-to-end loop")
    for ln in lanes[1:]:
        ln[0].close()
    link = (h2d + d2h) / (c_ms * 1e6)
    return {"value": job_throughput(T, world, e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": e_ms, "steps": Ke,
            "how": "piko_raster_forward_host (the C ABI with host buffers) per frame: the library copies "
                   "every input from pinned host memory, runs the forward pass and copies key and RGBA back; "
                   f"frames rotate over {nl} handles and {nl} streams so copies overlap the other frames' work",
            "sequential": {"value": job_throughput(T, world, seq_ms), "ms_per_step": seq_ms,
                           "how": "one frame at a time on one stream, L2 flushed between frames"},
            "copies_only": {"ms_per_step": c_ms, "gb_s": link, "frac_of_e2e_time": c_ms / e_ms,
                            "how": "the same frames' host<->device copies without the forward pass"},
            "bound": {"kind": "host link", "link_gb_s_measured": link,
                      "floor_ms": c_ms, "frac_of_floor": c_ms / e_ms,
                      "note": "each frame moves its inputs in and its 8-byte key plus float32 RGBA out; the "
                              "copies alone take copies_only.ms_per_step, which bounds this number"}}


def bin_sweep(args, ctx, scene, ds) -> dict:
    """Forward time of the headline workload at every bin size (8, 16, 32, 64)
    under the hardware and dynamic schedules (the workload's bin-size sweep),
    and under the fused (no tiling) and unfused (one kernel per stage)
    mappings of the same pipeline."""
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import Framebuffer, Rasterizer
    out = {}
    K = args.steps
    cands = [(b, sched) for b in (8, 16, 32, 64) for sched in ("hardware", "dynamic")]
    cands += [(16, "fused"), (16, "unfused")]  # the other two mappings (bins unused)
    for b, sched in cands:
        r = Rasterizer(scene.width, scene.height, b, b, sched)
        if args.perspective:
            r.set_option(L.PIKO_OPT_PERSPECTIVE, 1)
        fb = Framebuffer.allocate(scene.width, scene.height, scene.shade_mode)
        stats, covered = size_and_count(r, ds, fb)
        step_ms, stage_ms = time_forward(ctx, r, ds, fb, K, args.warmup)
        ms = sum(step_ms) / K
        rec = {"ms_per_step": ms, "value": scene.num_triangles / (ms * 1e-3) / 1e6}
        if sched in ("fused", "unfused"):
            # stage boundaries: raster, shading (unfused: fragment shader), depth test, composite
            rec["stage_ms"] = {n: float(stage_ms[:, i].mean()) for i, n in
                               enumerate(["vertex", "raster", "shade", "depth", "composite"])}
            out[sched] = rec
        else:
            rec.update({"process_ms": float(stage_ms[:, 4].mean()), "bin_entries": stats["bin_entries"]})
            out[f"{b}x{b} {sched}"] = rec
        r.close()
    return out


def measure_random256(args, ctx) -> dict:
    """256x256, 1,000 random triangles of 40-px radius, Gouraud, 16x16 bins,
    static schedule: a small frame, bound by launch latency."""
    from paper_1404_6293_gb300 import scenes as S
    from paper_1404_6293_gb300.raster import DeviceScene, Framebuffer, Rasterizer
    scene = S.random_triangles()
    r = Rasterizer(scene.width, scene.height, 16, 16, "static")
    ds = DeviceScene.from_host(scene)
    fb = Framebuffer.allocate(scene.width, scene.height, scene.shade_mode)
    stats, covered = size_and_count(r, ds, fb)
    K = args.steps
    m0 = ctx.clocks.mark()
    step_ms, stage_ms = time_forward(ctx, r, ds, fb, K, args.warmup)
    clk = ctx.clocks.summary(m0)
    if r.status()[0] != 0:
        raise RuntimeError("status error in the 256x256 loop")
    ms = sum(step_ms) / K
    proc_ms = float(stage_ms[:, 4].mean())
    rec = {"workload": "random triangles 256x256, 1,000 triangles of 40-px radius, Gouraud, 16x16 bins, static",
           "value": scene.num_triangles / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms,
           "shaded_gfrag_s": covered / (ms * 1e-3) / 1e9,
           "rasterized_gfrag_s": stats["fragments"] / (ms * 1e-3) / 1e9,
           "stage_ms": {n: float(stage_ms[:, i].mean()) for i, n in
                        enumerate(["vertex", "setup_count", "scan", "scatter", "process"])},
           "work": {**stats, "covered_pixels": covered},
           "roofline": process_roofline(ctx, scene, stats, proc_ms, clk), "clocks": clk,
           "gpu_launches": forward_launches(scene.width, scene.height, 16, 16) * K,
           "parity": "keys bit-exact, colour <= 1e-5 vs the oracle (tests/test_gpu_parity.py)"}
    if not args.no_cpu_baseline:
        import oracle
        cb = cpu_baseline(scene, args.config_cpu_seconds, single_seconds=1.0)
        t0 = time.perf_counter()
        key, _ = oracle.raster_brute(scene)
        oracle.shade(scene, key)
        dt = time.perf_counter() - t0
        cb["brute_force_single_thread"] = {"value": scene.num_triangles / dt / 1e6, "unit": UNIT,
                                           "sample": f"one full frame, every pixel against every triangle on "
                                                     f"one thread, {dt:.3f} s"}
        rec["cpu_baseline"] = cb
    r.close()
    return rec


def measure_reyes(args, ctx) -> dict:
    """The Reyes Sample stage on this path: micropolygon grids (256 Bezier
    patches diced to about half-pixel quads, two triangles each, 1024 x 768)
    sampled at pixel centres with the Sample stage's 32 x 32 bins and a
    diffuse (Lambert) Shade; the 16 x 16 hardware-scheduled launch beside it."""
    from paper_1404_6293_gb300 import scenes as S
    from paper_1404_6293_gb300.raster import DeviceScene, Framebuffer, Rasterizer
    scene = S.reyes_grids()
    ds = DeviceScene.from_host(scene)
    K = args.steps
    runs = {}
    for bins, sched in ((32, "dynamic"), (16, "hardware")):
        r = Rasterizer(scene.width, scene.height, bins, bins, sched)
        fb = Framebuffer.allocate(scene.width, scene.height, scene.shade_mode)
        stats, covered = size_and_count(r, ds, fb)
        m0 = ctx.clocks.mark()
        step_ms, stage_ms = time_forward(ctx, r, ds, fb, K, args.warmup)
        clk = ctx.clocks.summary(m0)
        if r.status()[0] != 0:
            raise RuntimeError("status error in the micropolygon loop")
        runs[(bins, sched)] = (sum(step_ms) / K, stage_ms, stats, covered, clk)
        r.close()
    ms, stage_ms, stats, covered, clk = runs[(32, "dynamic")]
    proc_ms = float(stage_ms[:, 4].mean())
    rec = {"workload": f"Reyes Sample: {scene.num_triangles} micropolygon triangles (256 bicubic patches diced to "
                       "~0.5-px quads), 1024x768, Lambert, 32x32 bins, dynamic",
           "value": scene.num_triangles / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms,
           "micropolygons_per_s": scene.num_triangles / 2 / (ms * 1e-3),
           "shaded_gfrag_s": covered / (ms * 1e-3) / 1e9,
           "stage_ms": {n: float(stage_ms[:, i].mean()) for i, n in
                        enumerate(["vertex", "setup_count", "scan", "scatter", "process"])},
           "work": {**stats, "covered_pixels": covered},
           "roofline": process_roofline(ctx, scene, stats, proc_ms, clk),
           "bins_16x16_hardware": {"ms_per_step": runs[(16, "hardware")][0],
                                   "value": scene.num_triangles / (runs[(16, "hardware")][0] * 1e-3) / 1e6},
           "clocks": clk, "gpu_launches": forward_launches(scene.width, scene.height, 32, 32) * K,
           "parity": "keys bit-exact, colour <= 1e-5 vs the oracle at this size (tests/test_gpu_reyes.py)"}
    if not args.no_cpu_baseline:
        rec["cpu_baseline"] = cpu_baseline(scene, args.config_cpu_seconds, single_seconds=2.0)
    return rec


def measure_deferred(args, ctx) -> dict:
    """Power-law 1080p (500k triangles, area pdf ~ a^-2), G-buffer forward
    then the 64-point-light pass."""
    import numpy as np
    import torch

    from paper_1404_6293_gb300 import scenes as S
    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300.raster import DeviceScene, Framebuffer, Rasterizer
    scene = S.power_law_triangles()
    lights = torch.from_numpy(S.point_lights(scene.width, scene.height, 64)).cuda()
    bins = args.deferred_bins
    r = Rasterizer(scene.width, scene.height, bins, bins, args.deferred_schedule)
    if args.small_px:
        r.set_option(L.PIKO_OPT_SMALL_TRI_PIXELS, args.small_px)
    if args.threads:
        r.set_option(L.PIKO_OPT_THREADS_PER_TILE, args.threads)
    ds = DeviceScene.from_host(scene)
    fb = Framebuffer.allocate(scene.width, scene.height, scene.shade_mode)
    out = torch.empty((scene.height, scene.width, 4), dtype=torch.float32, device="cuda")
    stats, covered = size_and_count(r, ds, fb)
    K = args.steps
    for _ in range(args.warmup):
        ctx.flush.zero_()
        r.forward(ds, fb)
        r.deferred_light(fb, lights, out)
    recs = []
    torch.cuda.synchronize()
    m0 = ctx.clocks.mark()
    for _ in range(K):
        ctx.flush.zero_()
        st = [ctx.event() for _ in range(L.PIKO_NUM_STAGE_EVENTS)]
        end = ctx.event()
        r.set_stage_events(st)
        r.forward(ds, fb)
        r.deferred_light(fb, lights, out)
        end.record(ctx.stream)
        recs.append((st, end))
    torch.cuda.synchronize()
    clk = ctx.clocks.summary(m0)
    if r.status()[0] != 0:
        raise RuntimeError("status error in the deferred loop")
    fwd = np.array([s[0].elapsed_time(s[5]) for s, _ in recs])
    light = np.array([s[5].elapsed_time(e) for s, e in recs])
    proc = np.array([s[4].elapsed_time(s[5]) for s, _ in recs])
    ms = float((fwd + light).mean())
    lt = float(light.mean()) * 1e-3
    light_ops = 30 * covered * 64
    alu_peak = ctx.alu_peak(clk)
    light_bytes = scene.width * scene.height * (8 + 8 + 8 + 16)
    rec = {"workload": "power-law 1920x1080, 500k triangles (area pdf ~ a^-2 on 1 px .. 1/4 screen), G-buffer "
                       f"+ 64 point lights, {bins}x{bins} bins, {args.deferred_schedule}",
           "value": scene.num_triangles / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms,
           "shaded_gfrag_s": covered / (ms * 1e-3) / 1e9,
           "rasterized_gfrag_s": stats["fragments"] / (ms * 1e-3) / 1e9,
           "forward_ms": float(fwd.mean()), "process_ms": float(proc.mean()), "light_pass_ms": float(light.mean()),
           "light_gpixlights_s": covered * 64 / lt / 1e9, "work": {**stats, "covered_pixels": covered},
           "roofline": process_roofline(ctx, scene, stats, float(proc.mean()), clk),
           "light_roofline": {"kernel": "k_deferred_light", "bound": "alu", "achieved": light_ops / lt / 1e9,
                              "peak": alu_peak, "unit": "Gop/s", "frac": light_ops / lt / 1e9 / alu_peak,
                              "hbm_frac": light_bytes / lt / 1e9 / ctx.hbm,
                              "ops": "30 thread-ops per (covered pixel, light)"},
           "clocks": clk, "gpu_launches": 6 * K,
           "parity": "keys bit-exact, G-buffer within one binary16 step, light pass <= 1e-5 vs the oracle "
                     "(tests/test_gpu_parity.py, tests/test_gpu_full_size.py)"}
    rec["exact_bins"] = exact_bins_record(ctx, scene, ds, bins, args.deferred_schedule, K, args.warmup, args.threads)
    if not args.no_cpu_baseline:
        import oracle
        lt_host = lights.cpu().numpy()

        def light_pass(key, g):
            oracle.light_pass(key, g[0], g[1], lt_host)
        rec["cpu_baseline"] = cpu_baseline(scene, args.config_cpu_seconds, extra=light_pass, single_seconds=2.0,
                                           what="bounding-box oracle, float64 G-buffer and 64-light pass")
    r.close()
    return rec


def measure_sphere(args, ctx) -> dict:
    """64 views at 512x512 of a 99.5k-triangle sphere, forward + L2-loss
    backward (colour, normal, light): one forward_batch and one
    backward_batch, each replayed from a CUDA graph."""
    import dataclasses

    import numpy as np
    import torch

    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300 import scenes as S
    from paper_1404_6293_gb300.raster import DeviceScene, Framebuffer, Rasterizer
    stream = ctx.stream
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
    neg2_tgt = tgt * -2.0  # the loss gradient 2 (rgba - target) as one elementwise pass
    fbs = [Framebuffer(key_all[v], rgba_all[v]) for v in range(nv)]
    gviews = [g_all[v] for v in range(nv)]
    dc = torch.zeros_like(ds.color)
    dn = torch.zeros_like(ds.normal)
    dl = torch.zeros_like(ds.light_dir)
    bins, scheds = [(16, 16)] * nv, ["dynamic"] * nv
    rb = Rasterizer(W, H, 16, 16)
    if args.perspective:
        rb.set_option(L.PIKO_OPT_PERSPECTIVE, 1)
    rb.forward_batch(views, fbs, bins, scheds)
    assert rb.status()[0] == 0
    rb.set_option(L.PIKO_OPT_CHECK_CAPACITY, 0)
    covered = int((key_all != -1).sum().item())

    def fwd_pass():
        rb.forward_batch(views, fbs, bins, scheds)

    def loss_pass():
        torch.add(neg2_tgt, rgba_all, alpha=2.0, out=g_all)

    def bwd_pass():
        dc.zero_(); dn.zero_(); dl.zero_()
        rb.backward_batch(views, fbs, gviews, [dc] * nv, [dn] * nv, [dl] * nv)

    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        for _ in range(2):
            fwd_pass(); loss_pass(); bwd_pass()
    stream.wait_stream(side)
    torch.cuda.synchronize()
    gf, gl, gb = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.graph(gf):
        fwd_pass()
    with torch.cuda.graph(gl):
        loss_pass()
    with torch.cuda.graph(gb):
        bwd_pass()
    torch.cuda.synchronize()
    K = args.steps
    for _ in range(args.warmup):
        ctx.flush.zero_()
        gf.replay(); gl.replay(); gb.replay()
    evs = [(ctx.event(), ctx.event(), ctx.event(), ctx.event()) for _ in range(K)]
    torch.cuda.synchronize()
    m0 = ctx.clocks.mark()
    for s, f, l, e in evs:
        ctx.flush.zero_()
        s.record(stream)
        gf.replay()
        f.record(stream)
        gl.replay()
        l.record(stream)
        gb.replay()
        e.record(stream)
    torch.cuda.synchronize()
    clk = ctx.clocks.summary(m0)
    assert rb.status()[0] == 0
    fwd = np.array([s.elapsed_time(f) for s, f, _, _ in evs])
    lossg = np.array([f.elapsed_time(l) for _, f, l, _ in evs])
    bwd = np.array([l.elapsed_time(e) for _, _, l, e in evs])
    ms = float((fwd + lossg + bwd).mean())
    T = nv * sph.num_triangles
    V = sph.num_vertices
    bw_bytes = nv * W * H * (8 + 16) + V * (16 + 12 * 2) + nv * V * 12 * 2
    bt = float(bwd.mean()) * 1e-3
    rec = {"workload": "sphere 99.5k triangles, 64 views 512x512, forward + L2-loss backward (colour, normal, light)",
           "value": T / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms,
           "shaded_gfrag_s": covered / (ms * 1e-3) / 1e9,
           "how": "the 64 views as one forward_batch, the loss gradient (one elementwise torch op) and one "
                  "backward_batch (16x16 bins, dynamic), each replayed from its own CUDA graph",
           "forward_ms": float(fwd.mean()), "loss_gradient_ms": float(lossg.mean()),
           "backward_ms": float(bwd.mean()), "covered_pixels": covered,
           "roofline": {"kernel": "k_batch_backward (64 views, with the gradient arrays' zeroing)", "bound": "hbm",
                        "achieved": bw_bytes / bt / 1e9, "peak": ctx.hbm, "unit": "GB/s",
                        "frac": bw_bytes / bt / 1e9 / ctx.hbm, "traffic": None,
                        "bytes": "24 B per pixel (key, dL/dRGBA) + 40 B per vertex read + 24 B per vertex per view "
                                 "of gradient updates"},
           "clocks": clk, "gpu_launches": 2 * K,
           "parity": "keys bit-exact, colour <= 1e-5, gradients <= 1e-4 rel vs the oracle on every view "
                     "(tests/test_gpu_full_size.py)"}
    if not args.no_cpu_baseline:
        import oracle
        sv = S.Scene(W, H, sph.pos, sph.tris, color=sph.color, normal=sph.normal, mvp=mvps[0],
                     light_dir=sph.light_dir, shade_mode=sph.shade_mode)
        tg0 = tgt[0].cpu().numpy()

        def backward(key, rgba):
            gg = np.zeros((H, W, 4))
            gg[..., :3] = 2 * (rgba[..., :3] - tg0[..., :3])
            oracle.backward(sv, key, gg, perspective=args.perspective)
        rec["cpu_baseline"] = cpu_baseline(sv, args.config_cpu_seconds, args.perspective, extra=backward,
                                           single_seconds=2.0,
                                           what="bounding-box oracle, float64 shading and gradients, one view")
    rb.close()
    return rec


def measure_batch(args, ctx) -> dict:
    """256 scenes (1k-200k triangles, 256^2-1024^2): plain per-scene loop of
    forward + backward (16x16 bins, static) against the autotuned batch,
    forward_batch + backward_batch replayed from one CUDA graph."""
    import numpy as np
    import torch

    from paper_1404_6293_gb300 import _lib as L
    from paper_1404_6293_gb300 import scenes as S
    from paper_1404_6293_gb300.autotune import Autotuner
    from paper_1404_6293_gb300.raster import DeviceScene, Framebuffer, Rasterizer

    stream = ctx.stream
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
    # the loss is sum over pixels of |rgb - target|^2; its gradient 2 (rgba -
    # target) is one elementwise pass, g = 2 rgba + (-2 target) (the backward
    # reads only the rgb part of g)
    neg2_target = target * -2.0
    g_all = torch.empty((P, 4), device="cuda")

    def loss_grad(rgba):
        torch.add(neg2_target, rgba, alpha=2.0, out=g_all)
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
        loss_grad(rgba_p)
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

    def batched_fwd():
        rb.forward_batch(ds, fbs_b, bins, scheds)

    def batched_loss():
        loss_grad(rgba_b)

    def batched_bwd():
        dc_b.zero_(); dn_b.zero_(); dl_b.zero_()
        rb.backward_batch(ds, fbs_b, gviews, dcv_b, dnv_b, dlv_b)

    for _ in range(2):
        batched_fwd(); batched_loss(); batched_bwd()
    torch.cuda.synchronize()
    gf, gl, gb = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.graph(gf):
        batched_fwd()
    with torch.cuda.graph(gl):
        batched_loss()
    with torch.cuda.graph(gb):
        batched_bwd()
    torch.cuda.synchronize()

    def timed(steps, K, W):
        """Mean ms of each part of a step (events between the parts)."""
        for _ in range(W):
            ctx.flush.zero_()
            for f in steps:
                f()
        torch.cuda.synchronize()
        tot = [0.0] * len(steps)
        for _ in range(K):
            ctx.flush.zero_()
            ev = [ctx.event() for _ in range(len(steps) + 1)]
            ev[0].record(stream)
            for j, f in enumerate(steps):
                f()
                ev[j + 1].record(stream)
            ev[-1].synchronize()
            for j in range(len(steps)):
                tot[j] += ev[j].elapsed_time(ev[j + 1])
        return [t / K for t in tot]

    m0 = ctx.clocks.mark()
    ms_plain = sum(timed([plain_step], args.steps, args.warmup))
    m1 = ctx.clocks.mark()
    f_ms, l_ms, b_ms = timed([gf.replay, gl.replay, gb.replay], args.steps, args.warmup)
    ms_batch = f_ms + l_ms + b_ms
    clk = ctx.clocks.summary(m1)
    clk["plain_loop"] = {k: v for k, v in ctx.clocks.summary(m0, m1).items() if k in ("sm_mhz", "samples", "reasons")}
    assert rb.status()[0] == 0
    same_keys = bool(torch.equal(key_p, key_b))
    gdiff = max(float((dc_p - dc_b).abs().max()), float((dn_p - dn_b).abs().max()), float((dl_p - dl_b).abs().max()))
    gscale = max(float(dc_p.abs().max()), float(dn_p.abs().max()), float(dl_p.abs().max()))
    covered = int((key_b != -1).sum().item())
    n_static = sum(1 for x in scheds if x == "static")
    # must-move bytes of the batched backward: 24 B per pixel (key and dL/dRGBA
    # read), per vertex 16 B position + 12 B colour + 12 B normal read and two
    # gradient arrays of 12 B read and written
    nrm = sum(1 for s in host if s.normal is not None)
    bw_bytes = P * 24 + VT * (16 + 12 + 12 + 48)
    rec = {"workload": f"{n} scenes, 1k-200k triangles (log-uniform), 256^2-1024^2, random + heightfield, "
                       "forward + L2 backward",
           "value": T / (ms_batch * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms_batch,
           "scenes": n, "triangles": T, "pixels": P, "scenes_with_normals": nrm,
           "shaded_gfrag_s": covered / (ms_batch * 1e-3) / 1e9,
           "plain": {"value": T / (ms_plain * 1e-3) / 1e6, "ms_per_step": ms_plain,
                     "how": "per-scene piko_raster_forward then piko_raster_backward, 16x16 static"},
           "batched": {"value": T / (ms_batch * 1e-3) / 1e6, "ms_per_step": ms_batch,
                       "forward_ms": f_ms, "loss_gradient_ms": l_ms, "backward_ms": b_ms,
                       "how": ("forward_batch (one persistent cooperative launch)" if args.batch_launch ==
                               "persistent" else "forward_batch (one launch per phase)") + ", the loss gradient "
                              "(one elementwise torch op) and backward_batch (with the gradient arrays' zeroing), "
                              "each replayed from its own CUDA graph",
                       "autotune_s": tune_s, "static_scenes": n_static,
                       "bins_used": sorted(set(f"{a}x{b}" for a, b in bins)),
                       "autotune": {"choice": tune_report["choice"], "classes": tune_report["classes"],
                                    "per_class_forward_ms": tune_report["per_class_ms"],
                                    "best_uniform_forward_ms": tune_report["best_uniform_ms"],
                                    "uniform_forward_ms": {f"{u['bin'][0]}x{u['bin'][1]} {u['schedule']}": u["ms"]
                                                           for u in tune_report["uniform"]}}},
           "speedup_batched_over_plain": ms_plain / ms_batch,
           "roofline": {"kernel": "k_batch_backward (with the gradient arrays' zeroing)", "bound": "hbm",
                        "achieved": bw_bytes / (b_ms * 1e-3) / 1e9, "peak": ctx.hbm, "unit": "GB/s",
                        "frac": bw_bytes / (b_ms * 1e-3) / 1e9 / ctx.hbm, "traffic": None,
                        "algorithmic_bytes": bw_bytes},
           "parity": {"keys_bit_identical_plain_vs_batched": same_keys, "grad_max_abs_diff": gdiff,
                      "grad_scale": gscale,
                      "oracle": "every scene's keys bit-exact and colour <= 1e-5 vs the oracle "
                                "(tests/test_gpu_full_size.py)"},
           "clocks": clk, "gpu_launches": (2 if args.batch_launch == "persistent" else 6) * args.steps,
           "gpu_launches_plain": sum(forward_launches(s.width, s.height, 16, 16) + 2 for s in host) * args.steps}
    if not args.no_cpu_baseline:
        import oracle
        hc = host_cpu()
        # a bounded sample: whole scenes in order until the time budget is spent
        t0 = time.perf_counter()
        done_t = 0
        k = 0
        while k < n and time.perf_counter() - t0 < args.config_cpu_seconds:
            sc = host[k]
            key, _ = oracle.raster_bbox(sc, threads=hc["cores"])
            rgba = oracle.shade(sc, key)
            tg = target[po[k]:po[k + 1]].view(sc.height, sc.width, 4).cpu().numpy()
            gg = np.zeros((sc.height, sc.width, 4))
            gg[..., :3] = 2 * (rgba[..., :3] - tg[..., :3])
            oracle.backward(sc, key, gg)
            done_t += sc.num_triangles
            k += 1
        dt = time.perf_counter() - t0
        rec["cpu_baseline"] = {"value": done_t / dt / 1e6, "unit": UNIT, "cores": hc["cores"],
                               "cpu_model": hc["cpu_model"], "kind": "oracle",
                               "sample": f"the first {k} of {n} scenes ({done_t} triangles): bounding-box oracle, "
                                         f"float64 shading and gradients on {hc['cores']} threads, {dt:.2f} s"}
    for h in handles.values():
        h.close()
    rb.close()
    return rec


def run_single_workload(args):
    """One of the other configurations as the line's value (for profiling
    and sweeps); the default run attaches them all under ``configs``."""
    import torch
    torch.cuda.set_device(0)
    clocks = ClockSampler(0)
    ctx = Ctx(clocks)
    fn = {"random256": measure_random256, "deferred": measure_deferred, "sphere": measure_sphere,
          "batch": measure_batch, "reyes": measure_reyes}[args.workload]
    rec = fn(args, ctx)
    clocks.close()
    line = {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic",
            "dtype": "int64+f32", "config": {"workload": rec.pop("workload"),
                                             "l2": "flushed between steps (256 MiB write)"}}
    line.update(rec)
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--bins", type=int, default=32,
                    help="bin size of the heightfield line (32: the fastest of the bin-size x schedule sweep)")
    ap.add_argument("--bin-h", type=int, default=0, help="bin height of the heightfield line (0: square bins)")
    ap.add_argument("--schedule", default="hardware", choices=["static", "dynamic", "hardware", "fused", "unfused"],
                    help="tile schedule of the heightfield line (hardware: one CTA per tile)")
    ap.add_argument("--threads", type=int, default=0, help="Process CTA size (0: library default)")
    ap.add_argument("--perspective", action="store_true",
                    help="heightfield and sphere workloads: perspective-correct attributes (PIKO_OPT_PERSPECTIVE)")
    ap.add_argument("--autotune", action="store_true",
                    help="heightfield workload: bin size, schedule and threads per bin from the autotuner")
    ap.add_argument("--small-px", type=int, default=0,
                    help="largest box (pixels inside a tile) one thread rasterizes; larger boxes take a warp "
                         "(0: library default)")
    ap.add_argument("--exact-bins", type=int, default=0, choices=[0, 1],
                    help="heightfield workload: AssignBin's exact overlap test instead of bounding-box bins")
    ap.add_argument("--deferred-bins", type=int, default=16)
    ap.add_argument("--deferred-schedule", default="hardware", choices=["static", "dynamic", "hardware", "fused", "unfused"])
    ap.add_argument("--batch-scenes", type=int, default=256)
    ap.add_argument("--batch-bins", type=int, default=0, help="batch workload: one square bin size for all scenes "
                    "instead of the autotuner's choice (0: autotune)")
    ap.add_argument("--batch-schedule", default="dynamic", choices=["static", "dynamic"])
    ap.add_argument("--batch-launch", default="persistent", choices=["persistent", "per-phase"],
                    help="batch workload: one cooperative launch, or one launch per phase (for launch lists)")
    ap.add_argument("--workload", default="heightfield",
                    choices=["heightfield", "random256", "deferred", "sphere", "batch", "reyes"],
                    help="heightfield: the headline line (with every other configuration under 'configs'); "
                         "the others: that configuration alone as the line")
    ap.add_argument("--no-configs", action="store_true", help="headline line only (no bin sweep, no other configs)")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-lanes", type=int, default=3, help="handles/streams the end-to-end frames rotate over")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--config-cpu-seconds", type=float, default=4.0,
                    help="oracle time budget (all cores) of each further configuration's cpu_baseline")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        sys.exit(run_reference(args))
    sys.exit(run_ours(args) if args.workload == "heightfield" else run_single_workload(args))


if __name__ == "__main__":
    main()
