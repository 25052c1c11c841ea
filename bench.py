#!/usr/bin/env python
"""Throughput of the Splotch hot path on GB300 (one JSON line on stdout).

A step is one full frame of the hot path (raster + tile count, scan, scatter,
splat + final transform) over the resident synthetic particle set.  The default
workload is the two-species 100 M-particle frame at 2048^2 with FP16 attribute
storage and FP32 accumulation.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

Workloads: two_species_f16 (default), two_species_f32, two_species_small, clustered,
plain, two_species_vector_f16 (stars coloured from a per-particle RGB field), batched
(64 orbit views in one CUDA-graph plan), served (request stream), streamed (out of core
from host memory), ordered (absorption different from emission, depth-ordered transfer),
ordered_small (the same on the 10 M two-species frame: the small case for profiles).
The default run also measures the frame with FP32 storage, a 64-view batched plan and a
short served trace (see extras); --no-extras leaves them out.

Under torchrun (N > 1) every rank renders its own replica of the frame (the
path needs no collective for independent frames); the step time is the maximum
over ranks and the value counts the particles of all ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mparticles/s and frames/s at 1 GB300; served p50/p99 latency; % HBM roofline"
UNIT = "Mparticles/s"
L2_BYTES = 129 * 2 ** 20


def load_brightness():
    p = os.path.join(ROOT, "tests", "golden", "brightness.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


def make_workload(name: str):
    """(particle set, camera, storage, description)."""
    from paper_1606_04427_gb300 import synth
    beta = load_brightness()
    cache = os.environ.get("SPLOTCH_SYNTH_CACHE")
    if name == "two_species_f16" or name == "two_species_f32":
        ps = _cached(cache, "two_species", lambda: synth.two_species_set(70_000_000, 30_000_000, 2))
        cam = synth.front_camera(2048, 2048)
        storage = "f16" if name.endswith("f16") else "f32"
        b = beta.get("two_species", [1.0, 1.0])
    elif name == "two_species_vector_f16":
        # the same frame with the stars coloured from a per-particle RGB field
        ps = _cached(cache, "two_species", lambda: synth.two_species_set(70_000_000, 30_000_000, 2))
        ps = synth.with_vector_colour(ps, [1], 2)
        cam = synth.front_camera(2048, 2048)
        storage = "f16"
        b = beta.get("two_species", [1.0, 1.0])
    elif name == "two_species_small":
        ps = _cached(cache, "two_species_small", lambda: synth.two_species_set(7_000_000, 3_000_000, 2))
        cam = synth.front_camera(2048, 2048)
        storage = "f16"
        b = [v * 10 for v in beta.get("two_species", [0.1, 0.1])]
    elif name == "clustered":
        ps = _cached(cache, "clustered", lambda: synth.clustered_set(10_000_000, 1))
        cam = synth.front_camera(1024, 1024)
        storage = "f32"
        b = beta.get("clustered", [1.0])
    elif name == "plain":
        ps = synth.plain_set(100_000, 0)
        cam = synth.front_camera(256, 256)
        storage = "f32"
        b = beta.get("plain", [1.0])
    else:
        raise SystemExit(f"unknown workload {name}")
    return ps.with_brightness(b), cam, storage


def _cached(cache_dir, key, fn):
    from paper_1606_04427_gb300 import synth
    if not cache_dir:
        return fn()
    os.makedirs(cache_dir, exist_ok=True)
    path = os.path.join(cache_dir, key + ".npz")
    if os.path.exists(path):
        z = np.load(path, allow_pickle=False)
        nt = int(z["type_begin"].shape[0] - 1)
        return synth.ParticleSet(z["x"], z["y"], z["z"], z["h"], z["intensity"], z["type_begin"],
                                 [z[f"cmap{t}"] for t in range(nt)], z["brightness"], z["i_log"],
                                 z["i_min"], z["i_max"], key)
    ps = fn()
    np.savez(path, x=ps.x, y=ps.y, z=ps.z, h=ps.h, intensity=ps.intensity, type_begin=ps.type_begin,
             brightness=ps.brightness, i_log=ps.i_log, i_min=ps.i_min, i_max=ps.i_max,
             **{f"cmap{t}": c for t, c in enumerate(ps.cmaps)})
    return ps


# library kernels per frame (single view) and per plan launch (all views at once): count,
# chunk-base scan, tile scan, scatter, work-item order, splat (with the final transform)
KERNELS_PER_FRAME = 6


def attr_bytes(storage):
    return 4 if storage == "f32" else 2


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            # raw samples: SPLOTCH_CLOCK_LOG_DIR when set (kept beside other run output),
            # else the temporary directory
            d = os.environ.get("SPLOTCH_CLOCK_LOG_DIR") or tempfile.gettempdir()
            os.makedirs(d, exist_ok=True)
            self.path = os.path.join(d, f"clocks_bench_{os.getpid()}.csv")
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# Arithmetic peak of the FP32 pipe, from the unit counts of the part: 152 SMs x 128 FP32
# lanes x 2 flops per fused multiply-add x the maximum SM clock; the special-function
# units give 16 exponentials per SM per clock.
N_SM = 152
FP32_LANES_PER_SM = 128
SFU_PER_SM = 16
# Algorithmic arithmetic of one covered (particle, pixel) pair (Section 2.1):
# dx = px - X (1), d2 = dx*dx + dy2 (2), exponent argument d2 * (-1/sigma^2) (1),
# three channel updates a += e * w (6); plus one exponential.
SPLAT_FLOPS_PER_PAIR = 10

# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant
# kernel, from one ncu capture of the small case of the same workload (two_species_small:
# a tenth of the particles, the same image), scaled to the full launch by the tile records
# read (204374882 against 20443231; the image write does not scale); valid only while the
# kernel source hashes to the recorded digest, else reported as null.
TRAFFIC = {
    "two_species_f16": {"bytes_per_launch": round(353393408 * 204374882 / 20443231) + 22131968,
                        "digest": "f5162254d69553fc", "kernel": "k_splat_warp<4,2>", "tile": 16,
                        "source": "small-case capture scaled by records"},
}


def kernel_digest():
    import hashlib
    d = hashlib.sha256()
    for f in ("k_splat.cu", "splotch_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1606_04427_gb300", "csrc", f), "rb") as fh:
            d.update(fh.read())
    return d.hexdigest()[:16]


def work_units(name):
    p = os.path.join(ROOT, "tests", "golden", "work_units.json")
    if not os.path.exists(p):
        return None
    # the vector-colour frame has the geometry (particles, camera) of the plain one
    name = {"two_species_vector_f16": "two_species_f16"}.get(name, name)
    with open(p) as f:
        return json.load(f).get(name)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def cpu_baseline(ps, cam, storage, budget_s=15.0):
    """The FP64 oracle as it stands, on this host's cores, over a stride sample of the
    frame's particles (full image), scaled to Mparticles/s.  Two short probes separate
    the per-frame cost from the per-particle cost; the sample is then sized so that the
    timed render takes about ``budget_s`` seconds."""
    import oracle
    n = ps.n

    def timed(m):
        idx = np.arange(0, n, max(1, n // m))
        sub = ps.subset(idx)
        t0 = time.perf_counter()
        oracle.render(sub, cam, oracle.Params(), storage)
        return idx.shape[0], time.perf_counter() - t0

    m1, t1 = timed(max(1000, n // 2000))
    m2, t2 = timed(max(4000, n // 500))
    per = max((t2 - t1) / max(1, m2 - m1), 1e-10)
    target = int(min(n, max(m2, budget_s / per)))
    m, dt = timed(target)
    step = max(1, n // target)
    return {"value": m / dt / 1e6, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"every {step}th particle ({m} of {n}), full {cam.width}x{cam.height} frame, "
                      f"{storage} attributes, {dt:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    ps, cam, storage = make_workload(args.workload)
    n = ps.n
    step = max(1, n // args.ref_particles)
    sub = ps.subset(np.arange(0, n, step))
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.render(sub, cam, oracle.Params(), storage)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    val = sub.n / (ms / 1e3) / 1e6
    sample = f"every {step}th particle ({sub.n} of {n}) per step, full {cam.width}x{cam.height} frame"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args.workload, ps, cam, storage, None),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _timed_clocks(fn, steps, stream, local):
    """Run fn() steps times between CUDA events on `stream`, sampling clocks; returns
    (ms per step, clocks)."""
    import torch
    clocks = ClockSampler(local)
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        fn()
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    return ev0.elapsed_time(ev1) / steps, clk


def run_batched(args):
    """64 orbit views of 20 M clustered particles (FP16 storage) at 1024 x 1024 rendered
    by one plan replayed as a CUDA graph; tile and particles per CTA from the autotuner."""
    import torch
    from paper_1606_04427_gb300 import autotune, build, render, synth
    build.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    beta = load_brightness().get("batched", [1.0])
    ps = _cached(os.environ.get("SPLOTCH_SYNTH_CACHE"), "batched",
                 lambda: synth.clustered_set(20_000_000, 3)).with_brightness(beta)
    cams = synth.orbit_cameras(64, 1024, 1024)
    scene = render.Scene(ps, "f16")
    t0 = time.perf_counter()
    tuned = autotune.tune(scene, cams, tiles=(8, 16, 24, 32, 40, 48, 64), blocks=(0, 262144), repeats=2)
    sweep_s = time.perf_counter() - t0
    plan = render.Plan(scene, cams, tuned["params"], graph=True)
    out = plan.new_output()
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        plan.launch(out)
    plan.check()
    ms, clk = _timed_clocks(lambda: plan.launch(out), args.steps, stream, local)
    plan.check()
    info = plan.info()
    V, n = len(cams), ps.n
    units = work_units("batched_f16")
    peaks, _ = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = N_SM * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    line = {"metric": METRIC, "value": V * n / (ms * 1e-3) / 1e6, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched_orbit64_clustered20M_f16", "n_particles": n, "views": V,
                       "image": [1024, 1024], "storage": "f16", "accumulation": "f32",
                       "tile": info["tile"], "block_particles": tuned["params"].block_particles,
                       "l2": "inputs larger than L2: 0.20 GB of attributes + 0.81 GB of images per step"},
            "frames_per_s": V / (ms * 1e-3), "autotune": {"sweep_s": sweep_s, "table": tuned["table"]},
            "plan_device_bytes": info["device_bytes"], "gpu_launches": KERNELS_PER_FRAME * args.steps, "clocks": clk}
    if units:
        flops = units["pixel_pairs"] * SPLAT_FLOPS_PER_PAIR
        line["roofline"] = {"bound": "alu", "kernel": "whole batch (upper bound on the splat's time)",
                            "achieved": flops / (ms * 1e-3) / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                            "frac": flops / (ms * 1e-3) / 1e12 / fp32_peak, "traffic": None}
    print(json.dumps(line), flush=True)
    return 0


def run_served(args):
    """Poisson render requests over 8 resident FP16 clustered sets of 1 M to 200 M
    particles, images 512^2 to 4096^2, random cameras; continuous batching with admission
    by HBM footprint.  Saturated throughput first (all requests at once), then traces at
    0.5, 0.8 and 1.0 of it; latency is arrival to completion."""
    import torch
    from paper_1606_04427_gb300 import build, render, serve, synth
    build.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    beta = load_brightness().get("served")
    sizes = synth.served_set_sizes()
    cache = os.environ.get("SPLOTCH_SYNTH_CACHE")
    scenes = []
    for k, n in enumerate(sizes):
        ps = _cached(cache, f"served{k}", lambda n=n, k=k: synth.clustered_set(n, 4 + k))
        scenes.append(render.Scene(ps.with_brightness([beta[k]] if beta else [1.0]), "f16"))
        del ps
    rng = np.random.default_rng(4)
    nreq = args.served_requests
    srv = serve.Server(scenes, slots=args.slots)
    try:
        warm = synth.poisson_requests(rng, 16, 1e6, len(scenes))
        srv.run_trace(warm)
        burst = synth.poisson_requests(rng, nreq, 1e9, len(scenes))
        sat = srv.run_trace(burst)
        res = {"saturated": sat}
        for lam in (0.5, 0.8, 1.0):
            reqs = synth.poisson_requests(rng, nreq, lam * sat["requests_per_s"], len(scenes))
            res[f"lambda_{lam}"] = srv.run_trace(reqs)
        errors = list(srv.errors)
        peak = srv.peak_reserved
    finally:
        srv.close()
    r08 = res["lambda_0.8"]
    line = {"metric": METRIC, "value": sat["mparticles_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": nreq, "warmup": 16, "ms_per_step": 1e3 / sat["requests_per_s"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "served_8sets_1M-200M_f16", "set_sizes": sizes, "images": [512, 4096],
                       "slots": args.slots, "requests_per_trace": nreq, "storage": "f16"},
            "served": res, "p50_ms": r08["p50_ms"], "p99_ms": r08["p99_ms"], "peak_reserved_bytes": peak,
            "errors": errors[:5]}
    print(json.dumps(line), flush=True)
    return 0


def streamed_chunks(n, chunk):
    """Chunk sizes of splotch_render_streamed: from a sixth of `chunk` (at least 2^20),
    growing by 3/2 up to `chunk`."""
    out, b = [], 0
    step = max(1, min(chunk, max(chunk // 6, 1 << 20)))
    while b < n:
        out.append(min(step, n - b))
        b += out[-1]
        step = min(chunk, step + step // 2)
    return out


def run_streamed(args):
    """Out-of-core render of the two-species 100 M frame: the particles stay in page-locked
    host memory and are rendered in chunks (each chunk prepared on a side stream while the
    previous one renders).  Wall time of the synchronous call, which includes reading the
    2 GB of FP32 attributes from the host, plus the image read back to the host."""
    import torch
    from paper_1606_04427_gb300 import build, render
    build.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    ps, cam, storage = make_workload("two_species_f16")
    keep = []
    pinned = ps.with_brightness(ps.brightness)
    for k in ("x", "y", "z", "h", "intensity"):
        t = torch.from_numpy(np.ascontiguousarray(getattr(ps, k))).pin_memory()
        keep.append(t)
        setattr(pinned, k, t.numpy())
    out = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device="cuda")
    host_img = torch.empty_like(out, device="cpu").pin_memory()
    chunk = args.chunk or max(4_000_000, -(-ps.n // 3))
    for _ in range(args.warmup):
        render.render_streamed(pinned, cam, chunk, out=out, storage=storage)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        render.render_streamed(pinned, cam, chunk, out=out, storage=storage)
        host_img.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    clk = clocks.stop()
    ms = 1e3 * statistics.mean(times)
    n = ps.n
    line = {"metric": METRIC, "value": n / (ms * 1e-3) / 1e6, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "streamed_two_species100M_2048_f16", "n_particles": n, "chunk": chunk,
                       "chunks": len(streamed_chunks(n, chunk)), "image": [cam.width, cam.height], "storage": storage,
                       "inputs": "page-locked host memory, FP32, read during the timed call",
                       "l2": "inputs larger than L2: 2.0 GB of host attributes per step"},
            "ms_min": 1e3 * min(times),
            "e2e": {"value": n / (ms * 1e-3) / 1e6, "unit": UNIT, "h2d_bytes_per_step": n * 5 * 4,
                    "d2h_bytes_per_step": cam.width * cam.height * 12},
            "gpu_launches": None, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


ORDERED_ABSORB = [1.5, 0.3]  # gas absorbs more than it emits, stars less


def run_ordered(args):
    """Depth-ordered render of the two-species 100 M frame with absorption different from
    emission (gas 1.5, stars 0.3 times the emission): binning with depth keys, the stable
    radix sorts that put each tile list far to near, and the ordered transfer.  Inputs
    resident in HBM; each call is synchronous (it reads the status word), so the step time
    is the call's wall time, cross-checked with CUDA events on its stream."""
    import torch
    from paper_1606_04427_gb300 import build, render
    build.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    small = args.workload == "ordered_small"
    ps, cam, storage = make_workload("two_species_small" if small else "two_species_f16")
    tile = args.tile or render.default_tile(cam.width, cam.height)
    params = render.RenderParams(tile=tile)
    scene = render.Scene(ps, storage)
    out = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        scene.render_ordered(cam, ORDERED_ABSORB, params, out, stream)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    steps = max(1, args.steps // 4)
    t0 = time.perf_counter()
    ev0.record(stream)
    for _ in range(steps):
        scene.render_ordered(cam, ORDERED_ABSORB, params, out, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) * 1e3 / steps
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / steps
    host_img = torch.empty_like(out, device="cpu").pin_memory()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    scene.render_ordered(cam, ORDERED_ABSORB, params, out, stream)
    host_img.copy_(out, non_blocking=True)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t1) * 1e3
    n = ps.n
    line = {"metric": METRIC, "value": n / (ms * 1e-3) / 1e6, "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms, "wall_ms_per_step": wall, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(config_dict("ordered_two_species10M_2048_f16" if small else "ordered_two_species100M_2048_f16",
                                       ps, cam, storage, tile),
                           absorb=ORDERED_ABSORB),
            "e2e": {"value": n / (e2e_ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": cam.width * cam.height * 12,
                    "path": "particles resident in HBM; one call plus the image read back"},
            "gpu_launches": None, "clocks": clk}
    print(json.dumps(line), flush=True)
    scene.close()
    return 0


def extras(ps, cam, params, args, local):
    """Further parts of the metric, measured in the default run (one GPU, rank 0) so
    that they sit beside the headline number:
      two_species_f32  the same frame with FP32 attribute storage (the plain FP32
                       single-view path the reduced-precision form is compared with);
      batched          64 orbit views at 1024^2 in one plan replayed as a CUDA graph,
                       over 20 M particles drawn from the frame's clustered gas, FP16,
                       tile and particles per CTA from a short autotuner sweep;
      served           a Poisson request stream over 8 resident FP16 sets drawn from the
                       frame's clustered gas (1 M to 70 M particles, geometric), random
                       cameras, images 512^2 to 4096^2: saturated throughput, then a
                       trace at 0.8 of it with p50 / p99 latency (arrival to completion).
    The full-size batched and served workloads (their own 20 M set; sets up to 200 M)
    are bench.py --workload batched / served."""
    import torch
    from paper_1606_04427_gb300 import autotune, render, serve, synth
    res = {}
    stream = torch.cuda.current_stream()
    out = torch.empty((1, cam.height, cam.width, 3), dtype=torch.float32, device="cuda")

    # FP32 storage of the same frame
    sc32 = render.Scene(ps, "f32")
    for _ in range(3):
        sc32.render([cam], params, out)
    ms32, clk = _timed_clocks(lambda: sc32.render([cam], params, out), max(5, args.steps // 2), stream, local)
    sc32.close()
    res["two_species_f32"] = {"ms_per_step": ms32, "value": ps.n / (ms32 * 1e-3) / 1e6, "unit": UNIT,
                              "storage": "f32", "clocks": clk}

    # gas particles of the frame (the clustered species), in index order
    gas = np.arange(int(ps.type_begin[0]), int(ps.type_begin[1]))
    beta = load_brightness()

    def gas_subset(m, b):
        idx = gas[np.linspace(0, gas.shape[0] - 1, m).astype(np.int64)]
        sub = ps.subset(idx)
        one = synth.ParticleSet(sub.x, sub.y, sub.z, sub.h, sub.intensity, np.array([0, m], np.int64),
                                [sub.cmaps[0]], np.array([b], np.float32), sub.i_log[:1].copy(),
                                None if sub.i_min is None else sub.i_min[:1].copy(),
                                None if sub.i_max is None else sub.i_max[:1].copy(), "gas")
        return one

    # batched: 64 orbit views, one graph replay per step
    bset = gas_subset(min(20_000_000, gas.shape[0]), beta.get("batched", [1.0])[0])
    bscene = render.Scene(bset, "f16")
    cams = synth.orbit_cameras(64, 1024, 1024)
    t0 = time.perf_counter()
    tuned = autotune.tune(bscene, cams, tiles=(16, 32), blocks=(0, 262144), repeats=1, cache_path=None)
    sweep = time.perf_counter() - t0
    plan = render.Plan(bscene, cams, tuned["params"], graph=True)
    bout = plan.new_output()
    for _ in range(3):
        plan.launch(bout)
    plan.check()
    bsteps = 5
    msb, clkb = _timed_clocks(lambda: plan.launch(bout), bsteps, stream, local)
    plan.check()
    info = plan.info()
    res["batched"] = {"ms_per_step": msb, "frames_per_s": len(cams) / (msb * 1e-3),
                      "value": len(cams) * bset.n / (msb * 1e-3) / 1e6, "unit": UNIT, "views": len(cams),
                      "n_particles": bset.n, "image": [1024, 1024], "storage": "f16", "steps": bsteps,
                      "tile": info["tile"], "block_particles": tuned["params"].block_particles,
                      "autotune_sweep_s": sweep, "clocks": clkb}
    del plan, bout
    bscene.close()

    # served: saturated burst, then Poisson arrivals at 0.8 of the saturated rate
    sizes = [int(round(1e6 * (min(70e6, gas.shape[0]) / 1e6) ** (k / 7))) for k in range(8)]
    sb = beta.get("served")
    scenes = [render.Scene(gas_subset(m, sb[k] if sb else 1.0), "f16") for k, m in enumerate(sizes)]
    rng = np.random.default_rng(4)
    srv = serve.Server(scenes, slots=4)
    try:
        srv.run_trace(synth.poisson_requests(rng, 12, 1e6, len(scenes)))
        sat = srv.run_trace(synth.poisson_requests(rng, args.extra_requests, 1e9, len(scenes)))
        lam = 0.8 * sat["requests_per_s"]
        tr = srv.run_trace(synth.poisson_requests(rng, args.extra_requests, lam, len(scenes)))
        errors = list(srv.errors)
    finally:
        srv.close()
    for sc in scenes:
        sc.close()
    res["served"] = {"set_sizes": sizes, "storage": "f16", "slots": 4, "requests_per_trace": args.extra_requests,
                     "saturated": {k: sat[k] for k in ("requests_per_s", "mparticles_per_s", "p50_ms", "p99_ms")},
                     "lambda_per_s": lam, "lambda_frac_of_saturated": 0.8,
                     "requests_per_s": tr["requests_per_s"], "mparticles_per_s": tr["mparticles_per_s"],
                     "p50_ms": tr["p50_ms"], "p99_ms": tr["p99_ms"], "errors": errors[:3]}
    return res


def max_over_ranks(value: float) -> float:
    """The largest value over all ranks (the step time of the slowest GPU); a no-op
    outside torch.distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def config_dict(name, ps, cam, storage, tile):
    return {"workload": name, "n_particles": ps.n, "species": ps.n_types, "image": [cam.width, cam.height],
            "storage": storage, "accumulation": "f32", "tile": tile,
            "l2": f"inputs larger than L2: {ps.n * 5 * attr_bytes(storage) / 1e9:.2f} GB of attributes"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="two_species_f16")
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--ref-particles", type=int, default=2_000_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP32-storage, batched and served measurements of the default run")
    ap.add_argument("--extra-requests", type=int, default=160, help="requests per served trace in the default run")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--served-requests", type=int, default=400)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--chunk", type=int, default=0, help="out-of-core chunk (0: a quarter of the set, >= 4M)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "served":
        return run_served(args)
    if args.workload == "streamed":
        return run_streamed(args)
    if args.workload in ("ordered", "ordered_small"):
        return run_ordered(args)

    import torch
    from paper_1606_04427_gb300 import build, render

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    build.build()

    ps, cam, storage = make_workload(args.workload)
    params = render.RenderParams(tile=args.tile)
    tile = args.tile or render.default_tile(cam.width, cam.height)
    stream = torch.cuda.current_stream()
    scene = render.Scene(ps, storage)
    out = torch.empty((1, cam.height, cam.width, 3), dtype=torch.float32, device="cuda")

    for _ in range(args.warmup):
        scene.render([cam], params, out)
    torch.cuda.synchronize()

    # per-kernel durations (CUDA events on the launching stream, inside the library)
    kt = {"count": [], "scan": [], "scatter": [], "splat": []}
    sizes = None
    for _ in range(max(3, min(args.steps, 10))):
        scene.render([cam], render.RenderParams(tile=args.tile, timing=True), out)
        t = render.last_timing()
        for k in kt:
            kt[k].append(t[k])
        sizes = t
    kms = {k: statistics.mean(v) for k, v in kt.items()}

    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        scene.render([cam], params, out)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(ms)

    # end to end through the public API for particles held in host memory: the out-of-core
    # render reads the page-locked FP32 attributes chunk by chunk (the copy of chunk k + 1
    # overlapping the render of chunk k), then the image is read back to the host
    h2d = ps.n * 5 * 4
    d2h = cam.width * cam.height * 3 * 4
    e2e_ms = None
    e2e_chunk = args.chunk or max(4_000_000, -(-ps.n // 3))
    if args.e2e_steps > 0:
        pinned = ps.with_brightness(ps.brightness)
        keep = []
        for k in ("x", "y", "z", "h", "intensity"):
            t = torch.from_numpy(np.ascontiguousarray(getattr(ps, k))).pin_memory()
            keep.append(t)
            setattr(pinned, k, t.numpy())
        host_img = torch.empty((1, cam.height, cam.width, 3), dtype=torch.float32).pin_memory()
        e2e_times = []
        for k in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            render.render_streamed(pinned, cam, e2e_chunk, params, out=out[0], storage=storage)
            host_img.copy_(out, non_blocking=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            if k > 0:
                e2e_times.append(dt)
        e2e_ms = 1e3 * statistics.mean(e2e_times)

    if rank != 0:
        return 0

    peaks, peak_kind = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = N_SM * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12  # TFLOP/s
    b = attr_bytes(storage)
    n = ps.n
    P = sizes["pairs"]
    WH = cam.width * cam.height
    units = work_units(args.workload)
    # per-kernel algorithmic bytes: count reads x, y, z, h; scatter reads all five
    # attributes and writes a 16-byte record per pair; splat reads the records and writes
    # the image
    alg_bytes = {"count": n * 4 * b, "scatter": n * 5 * b + P * 16, "splat": P * 16 + WH * 12}
    kern = {}
    for k in ("count", "scatter"):
        gbs = alg_bytes[k] / (kms[k] * 1e-3) / 1e9
        kern[k] = {"bound": "hbm", "ms": kms[k], "bytes": alg_bytes[k], "achieved_gbs": gbs, "frac": gbs / hbm}
    splat = {"bound": "alu", "ms": kms["splat"], "bytes": alg_bytes["splat"],
             "achieved_gbs": alg_bytes["splat"] / (kms["splat"] * 1e-3) / 1e9}
    if units:
        flops = units["pixel_pairs"] * SPLAT_FLOPS_PER_PAIR
        splat.update({"pixel_pairs": units["pixel_pairs"], "flops": flops,
                      "achieved_tflops": flops / (kms["splat"] * 1e-3) / 1e12,
                      "exp_per_s": units["pixel_pairs"] / (kms["splat"] * 1e-3),
                      "sfu_frac": units["pixel_pairs"] / (kms["splat"] * 1e-3) / (N_SM * SFU_PER_SM * sm_max * 1e6)})
        splat["frac"] = splat["achieved_tflops"] / fp32_peak
    kern["splat"] = splat
    kern["scan"] = {"bound": "latency", "ms": kms["scan"]}
    dom = max(kms, key=lambda k: kms[k])
    digest = kernel_digest()
    tr = TRAFFIC.get(args.workload)
    traffic = (tr["bytes_per_launch"] if (tr and tr["digest"] == digest and dom == "splat" and tr["tile"] == tile)
               else None)
    frame_alg = n * 5 * b + WH * 12
    if dom == "splat" and "frac" in splat:
        roof = {"bound": "alu", "kernel": "k_splat", "achieved": splat["achieved_tflops"], "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": splat["frac"], "traffic": traffic,
                "peak_kind": f"derived FP32 pipe peak: {N_SM} SMs x {FP32_LANES_PER_SM} lanes x 2 flops x {sm_max:.0f} MHz",
                "algorithmic_flops_per_launch": splat["flops"], "flops_per_pixel_pair": SPLAT_FLOPS_PER_PAIR}
    else:
        roof = {"bound": kern[dom]["bound"], "kernel": dom, "achieved": kern[dom].get("achieved_gbs"), "peak": hbm,
                "unit": "GB/s", "frac": kern[dom].get("frac"), "traffic": traffic,
                "peak_kind": f"{peak_kind} copy bandwidth"}
    roof["kernel_digest"] = digest
    roof["frame_hbm_frac"] = frame_alg / (ms * 1e-3) / 1e9 / hbm
    roof["frame_hbm_note"] = (f"algorithmic bytes of the frame ({frame_alg / 1e9:.3f} GB: attributes + image) / "
                              f"step time, of {peak_kind} {hbm:.0f} GB/s")
    value = world * n / (ms * 1e-3) / 1e6
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_dict(args.workload, ps, cam, storage, tile),
            "frames_per_s": world * 1e3 / ms,
            "kernels_ms": kms, "kernels": kern, "pairs": P, "work_items": sizes["items"],
            "split_tiles": sizes["splits"], "work_units": units, "roofline": roof,
            "e2e": None if e2e_ms is None else {
                "value": n / (e2e_ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "path": f"splotch_render_streamed from page-locked host memory, "
                        f"{len(streamed_chunks(n, e2e_chunk))} chunks ramping up to {e2e_chunk} particles"},
            "gpu_launches": KERNELS_PER_FRAME * args.steps, "clocks": clk}
    if world == 1 and not args.no_extras:
        line.update(extras(ps, cam, params, args, local))
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(ps, cam, storage)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
