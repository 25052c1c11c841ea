"""Tile-size and particles-per-block autotuner for batched renders.

Section 3.2.3 sets tile size and thread-group parameters from scripted sweeps
of candidate values on the target hardware, read from a parameter file at run
time.  This module does the same on the GPU: for each candidate (tile edge,
particles per CTA) it builds a :class:`render.Plan` over the caller's views,
replays it a few times and keeps the fastest; results are cached in a JSON file
keyed by (particle-count bucket, image size, view count, storage, screen-radius
bucket), so a later run with a similar workload reads the choice instead of
sweeping again.
"""
from __future__ import annotations

import json
import math
import os
import time
from typing import Dict, Optional, Sequence

import numpy as np
import torch

from . import render

TILES = (8, 16, 24, 32, 40, 48, 64)
BLOCK_PARTICLES = (0, 65536, 262144, 1048576)  # 0 = library default (about four CTAs per SM)
MAX_TILES = 16384


def _radius_bucket(scene: render.Scene, cam) -> int:
    """log2 bucket of the median screen support radius of active particles."""
    r = scene.debug_raster(cam)
    R = r["R"][r["active"]]
    if R.numel() == 0:
        return -99
    med = float(R.float().median().item())
    return int(math.floor(math.log2(max(med, 1e-3)) * 2))


def cache_key(scene: render.Scene, cams: Sequence) -> str:
    c0 = cams[0]
    nb = int(math.floor(math.log2(max(1, scene.n)) * 2))
    return f"n{nb}_w{c0.width}_h{c0.height}_v{len(cams)}_{scene.storage}_r{_radius_bucket(scene, c0)}"


def time_plan(scene: render.Scene, cams: Sequence, params: render.RenderParams, repeats: int = 3,
              headroom: float = 1.25) -> float:
    """Mean milliseconds of one batched launch (graph replay) over ``repeats``."""
    plan = render.Plan(scene, cams, params, headroom=headroom, graph=True)
    try:
        out = plan.new_output()
        plan.launch(out)
        plan.check()
        s = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(repeats):
            plan.launch(out)
        e1.record(s)
        plan.check()
        return e0.elapsed_time(e1) / repeats
    finally:
        plan.close()


def tune(scene: render.Scene, cams: Sequence, base: Optional[render.RenderParams] = None,
         tiles: Sequence[int] = TILES, blocks: Sequence[int] = BLOCK_PARTICLES, repeats: int = 3,
         cache_path: Optional[str] = None, force: bool = False) -> Dict:
    """Pick (tile, block_particles) for this scene and these views.  Returns
    {"params": RenderParams, "ms": best, "table": [...], "cached": bool}."""
    base = base or render.RenderParams()
    key = cache_key(scene, cams)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    if not force and key in cache:
        hit = cache[key]
        p = render.RenderParams(**{**base.__dict__, "tile": hit["tile"], "block_particles": hit["block_particles"]})
        return {"params": p, "ms": hit["ms"], "table": hit.get("table", []), "cached": True, "key": key}
    W, H = cams[0].width, cams[0].height
    table = []
    best = None
    t_start = time.perf_counter()
    for T in tiles:
        if ((W + T - 1) // T) * ((H + T - 1) // T) > MAX_TILES:
            continue
        for bp in blocks:
            if bp and bp >= scene.n:
                continue
            p = render.RenderParams(**{**base.__dict__, "tile": T, "block_particles": bp})
            try:
                ms = time_plan(scene, cams, p, repeats)
            except Exception as e:  # a candidate the plan cannot hold is skipped
                table.append({"tile": T, "block_particles": bp, "error": str(e)[:120]})
                continue
            table.append({"tile": T, "block_particles": bp, "ms": ms})
            if best is None or ms < best[0]:
                best = (ms, T, bp)
    if best is None:
        raise RuntimeError("no autotune candidate could run")
    res = {"tile": best[1], "block_particles": best[2], "ms": best[0], "table": table,
           "sweep_s": time.perf_counter() - t_start}
    if cache_path:
        cache[key] = res
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    p = render.RenderParams(**{**base.__dict__, "tile": best[1], "block_particles": best[2]})
    return {"params": p, "ms": best[0], "table": table, "cached": False, "key": key}
