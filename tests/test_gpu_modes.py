"""Batched, served and sharded modes on the GPU, against the single-view path and the
oracle (needs a GB300)."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1606_04427_gb300 import _lib, autotune, build, render, serve, shard, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    assert torch.cuda.is_available()


def test_autotune_picks_a_candidate_and_caches_it(tmp_path):
    ps = synth.clustered_set(40000, 3, grid=64).with_brightness([0.05])
    sc = render.Scene(ps, "f16")
    cams = synth.orbit_cameras(4, 128, 96)
    cache = str(tmp_path / "tune.json")
    res = autotune.tune(sc, cams, tiles=(8, 16, 32), blocks=(0, 8192), repeats=2, cache_path=cache)
    assert res["params"].tile in (8, 16, 32) and not res["cached"]
    assert len([r for r in res["table"] if "ms" in r]) == 6
    again = autotune.tune(sc, cams, tiles=(8, 16, 32), blocks=(0, 8192), cache_path=cache)
    assert again["cached"] and again["params"].tile == res["params"].tile
    with open(cache) as f:
        assert res["key"] in json.load(f)
    # the tuned plan still renders the oracle's image
    plan = render.Plan(sc, cams, res["params"], graph=True)
    out = plan.new_output()
    plan.launch(out)
    plan.check()
    for v, cam in enumerate(cams):
        ref = oracle.final(oracle.render(ps, cam, oracle.Params(tile=res["params"].tile), "f16"))
        assert np.abs(out[v].cpu().numpy() - ref).max() <= 2e-3


def test_block_particles_do_not_change_the_image():
    ps = synth.clustered_set(50000, 7, grid=64).with_brightness([0.05])
    sc = render.Scene(ps, "f32")
    cam = synth.front_camera(160, 120)
    base = sc.render(cam).cpu().numpy()
    for bp in (1024, 5000, 40000):
        other = sc.render(cam, render.RenderParams(block_particles=bp)).cpu().numpy()
        assert np.abs(base - other).max() <= 1e-4


def _served_sets():
    rng = np.random.default_rng(12)
    sets = [synth.clustered_set(n, 20 + k, grid=32).with_brightness([b])
            for k, (n, b) in enumerate([(20000, 0.2), (60000, 0.07), (150000, 0.03)])]
    reqs = []
    t = 0.0
    for i in range(18):
        t += rng.exponential(0.002)
        cam = synth.random_camera(rng, sizes=(64, 96, 160, 256))
        reqs.append(synth.Request(int(rng.integers(0, 3)), cam, t))
    return sets, reqs


def test_server_result_alone_equals_result_in_the_mix():
    sets, reqs = _served_sets()
    scenes = [render.Scene(p, "f16") for p in sets]
    alone = [scenes[r.set_index].render(r.camera, render.RenderParams(sync=True)).cpu().numpy() for r in reqs]
    srv = serve.Server(scenes, slots=3, keep_images=True)
    try:
        st = srv.run_trace(reqs)
    finally:
        srv.close()
    assert not srv.errors, srv.errors
    assert st["requests"] == len(reqs) and st["p99_ms"] >= st["p50_ms"] > 0
    by_id = {d.request_id: d for d in srv.done}
    assert max(d.finish for d in srv.done) > 0
    for i, r in enumerate(reqs):
        img = by_id[i].image.cpu().numpy()
        assert np.abs(img - alone[i]).max() <= 1e-4, i
        ref = oracle.final(oracle.render(sets[r.set_index], r.camera, oracle.Params(), "f16"))
        assert np.abs(img - ref).max() <= 2e-3, i


def test_server_admission_by_footprint():
    """With a budget smaller than any request the server still drains the queue, one
    request in flight at a time; with a large budget requests overlap."""
    sets, reqs = _served_sets()
    scenes = [render.Scene(p, "f16") for p in sets]
    srv = serve.Server(scenes, slots=4, hbm_budget=1)
    inflight = []
    try:
        for r in reqs:
            srv.submit(r.set_index, r.camera)
        while srv.queue or srv.in_flight:
            inflight.append(srv.in_flight)
            torch.cuda.synchronize()
        srv.wait_all(timeout=120)
    finally:
        srv.close()
    assert len(srv.done) == len(reqs) and not srv.errors
    assert max(inflight) <= 1
    assert all(d.reserved_bytes > 0 for d in srv.done)


def test_server_reserves_exactly_what_the_library_allocates():
    """A budget just above the largest request's true footprint (count-phase workspace +
    tile lists + image, from the two-phase API): the queue drains without errors, the
    reservations never exceed the budget, and every request reserved exactly the bytes the
    library and its image took.  The frames still match the plain render."""
    sets, reqs = _served_sets()
    scenes = [render.Scene(p, "f16") for p in sets]
    foot = []
    for r in reqs:
        sc = scenes[r.set_index]
        f = sc.prepare(r.camera)
        assert f.fixed_bytes == sc.frame_fixed_bytes(r.camera)
        foot.append(f.fixed_bytes + f.var_bytes + r.camera.width * r.camera.height * 12)
        img = f.render()
        torch.cuda.synchronize()
        want = sc.render(r.camera, render.RenderParams(sync=True))
        assert torch.allclose(img, want, rtol=0, atol=1e-4)
        f.close()
    budget = max(foot) + (1 << 20)
    srv = serve.Server(scenes, slots=4, hbm_budget=budget)
    try:
        for r in reqs:
            srv.submit(r.set_index, r.camera)
        srv.wait_all(timeout=120)
    finally:
        srv.close()
    assert not srv.errors, srv.errors
    assert len(srv.done) == len(reqs)
    assert srv.peak_reserved <= budget, (srv.peak_reserved, budget)
    for d in srv.done:
        assert d.reserved_bytes == d.allocated_bytes == foot[d.request_id], d
    with pytest.raises(_lib.SplotchError):
        f = scenes[0].prepare(reqs[0].camera)
        f.render()
        f.render()  # a frame renders once


def test_shards_sum_to_the_whole_frame():
    """Linearity of the accumulation: rendering two particle shards and summing equals
    rendering all of them (the multi-GPU exchange, checked on one GPU)."""
    ps = synth.two_species_set(30000, 10000, 8, grid=32).with_brightness([0.05, 0.3])
    cam = synth.front_camera(120, 100)
    whole = render.Scene(ps, "f32").render(cam, render.RenderParams(accum=True))
    parts = [render.Scene(shard.shard_particles(ps, r, 3), "f32").render(cam, render.RenderParams(accum=True))
             for r in range(3)]
    summed = parts[0] + parts[1] + parts[2]
    assert torch.allclose(summed, whole, rtol=2e-5, atol=1e-7)
    shard.final_transform_(summed)
    ref = oracle.final(oracle.render(ps, cam))
    assert np.abs(summed.cpu().numpy() - ref).max() <= 1e-4


def test_concurrent_renders_of_different_image_sizes():
    """Host threads rendering different image sizes at once (each on its own stream):
    the kernels' per-launch shared-memory needs differ, and no launch may see another
    thread's setting.  Every image equals the same render made alone."""
    import threading
    ps = synth.clustered_set(60000, 9, grid=64).with_brightness([0.05])
    sc = render.Scene(ps, "f32")
    sizes = [(64, 48), (512, 512), (1024, 768), (200, 130), (2048, 1024), (96, 96)]
    cams = [synth.front_camera(w, h) for w, h in sizes]
    alone = [sc.render(c, render.RenderParams(sync=True)).cpu() for c in cams]
    errors, results = [], {}

    def work(k):
        try:
            st = torch.cuda.Stream()
            for rep in range(6):
                j = (k + rep) % len(cams)
                img = sc.render(cams[j], render.RenderParams(sync=True), stream=st)
                results[(k, rep)] = (j, img.cpu())
        except Exception as e:  # collected and asserted below
            errors.append(repr(e))

    threads = [threading.Thread(target=work, args=(k,)) for k in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=120)
    assert not errors, errors
    assert len(results) == 24
    for (k, rep), (j, img) in results.items():
        assert torch.abs(img - alone[j]).max().item() <= 1e-4, (k, rep, sizes[j])


def test_scene_from_page_locked_host_memory_equals_pageable():
    """Page-locked host inputs are read in place by the device; the scene renders the
    same image as one built from pageable copies of the same arrays."""
    ps = synth.two_species_set(30000, 10000, 6, grid=32).with_brightness([0.05, 0.3])
    cam = synth.front_camera(160, 120)
    pageable = render.Scene(ps, "f16").render(cam).cpu()
    pinned = ps.with_brightness(ps.brightness)
    keep = []
    for k in ("x", "y", "z", "h", "intensity"):
        t = torch.from_numpy(np.ascontiguousarray(getattr(ps, k))).pin_memory()
        keep.append(t)
        setattr(pinned, k, t.numpy())
    sc = render.Scene(pinned, "f16")
    got = sc.render(cam).cpu()
    assert torch.equal(got, pageable) or torch.abs(got - pageable).max().item() <= 1e-6
    ref = oracle.final(oracle.render(ps, cam, oracle.Params(), "f16"))
    assert np.abs(got.numpy() - ref).max() <= 2e-3


def _no_ranges(ps):
    out = ps.with_brightness(ps.brightness)
    out.i_min = None
    out.i_max = None
    return out


def test_streamed_render_equals_resident_render():
    """Out-of-core render in chunks that cut through a species boundary equals the render
    of the whole resident set (a sum over particles), for given and for computed intensity
    ranges, from pageable and from page-locked host arrays; and it matches the oracle."""
    ps = synth.two_species_set(30000, 10000, 11, grid=32).with_brightness([0.05, 0.3])
    cam = synth.front_camera(200, 150)
    whole = render.Scene(ps, "f32").render(cam).cpu()
    for chunk in (7000, 16384, 40000):
        got = render.render_streamed(ps, cam, chunk).cpu()
        assert torch.abs(got - whole).max().item() <= 1e-4, chunk
    free = _no_ranges(ps)
    whole_free = render.Scene(free, "f32").render(cam).cpu()
    got = render.render_streamed(free, cam, 9000).cpu()
    assert torch.abs(got - whole_free).max().item() <= 1e-4
    pinned = ps.with_brightness(ps.brightness)
    keep = []
    for k in ("x", "y", "z", "h", "intensity"):
        t = torch.from_numpy(np.ascontiguousarray(getattr(ps, k))).pin_memory()
        keep.append(t)
        setattr(pinned, k, t.numpy())
    got16 = render.render_streamed(pinned, cam, 12000, storage="f16").cpu().numpy()
    ref = oracle.final(oracle.render(ps, cam, oracle.Params(), "f16"))
    assert np.abs(got16 - ref).max() <= 2e-3
    acc = render.render_streamed(ps, cam, 8000, render.RenderParams(accum=True)).cpu()
    whole_acc = render.Scene(ps, "f32").render(cam, render.RenderParams(accum=True)).cpu()
    assert torch.allclose(acc, whole_acc, rtol=2e-5, atol=1e-7)


def _max_contributions(ps, cam):
    """Largest number of particles covering one pixel (the oracle's FP32 raster and the
    coverage rule d^2 < R^2), for the summation-order bound."""
    r = oracle.raster(ps, cam)
    a = r["active"]
    X, Y, R = (r[k][a].astype(np.float32) for k in ("X", "Y", "R"))
    cnt = np.zeros((cam.height, cam.width), np.int64)
    for x, y, rr in zip(X, Y, R):
        i0, i1 = max(0, int(np.ceil(x - rr - 0.5)) - 1), min(cam.width - 1, int(np.floor(x + rr - 0.5)) + 1)
        j0, j1 = max(0, int(np.ceil(y - rr - 0.5)) - 1), min(cam.height - 1, int(np.floor(y + rr - 0.5)) + 1)
        if i0 > i1 or j0 > j1:
            continue
        px = np.arange(i0, i1 + 1, dtype=np.float32) + np.float32(0.5)
        py = np.arange(j0, j1 + 1, dtype=np.float32) + np.float32(0.5)
        dx2 = (px - x) * (px - x)
        dy2 = (py - y) * (py - y)
        cnt[j0:j1 + 1, i0:i1 + 1] += (dy2[:, None] + dx2[None, :]) < rr * rr
    return int(cnt.max())


# A pixel's accumulation is a sum of n non-negative FP32 terms (Section 3.2.2: colour x
# scalar weight).  Without SPLOTCH_STABLE the order of the terms inside one chunk's part
# of a tile list may change from run to run (the reading that the summation order inside
# a pixel is free), and any order's FP32 sum lies within (n - 1) 2^-24 of the exact sum,
# relative; the tests below derive their bounds from that.
U32 = 2.0 ** -24


def test_additive_output_sums_renders():
    """SPLOTCH_OUT_ADD adds the accumulation to the output: two additive renders of the
    same frame give twice the accumulation, exactly with stable tile lists, and within the
    summation-order bound (4 (n - 1) + 2) 2^-24 relative without them."""
    ps = synth.clustered_set(30000, 12, grid=32).with_brightness([0.05])
    cam = synth.front_camera(128, 96)
    sc = render.Scene(ps, "f32")
    acc = sc.render(cam, render.RenderParams(accum=True, stable=True))
    out = torch.zeros_like(acc)
    sc.render(cam, render.RenderParams(add=True, stable=True), out)
    sc.render(cam, render.RenderParams(add=True, stable=True), out)
    assert torch.equal(out, 2 * acc)
    n = _max_contributions(ps, cam)
    rtol = (4 * (n - 1) + 2) * U32
    out.zero_()
    sc.render(cam, render.RenderParams(add=True), out)
    sc.render(cam, render.RenderParams(add=True), out)
    assert torch.allclose(out, 2 * acc, rtol=rtol, atol=0.0), (n, rtol)


@pytest.mark.parametrize("T", [8, 16, 24, 32, 40, 64])
def test_renders_are_bitwise_reproducible(T):
    """With stable tile lists the same frame rendered again, with other work in between
    and a different number of particle chunks, gives the same bits: every tile list is in
    ascending particle index and the slices of a split tile merge exactly, so no
    summation order depends on which CTA or warp runs first.  Without them a render stays
    within the summation-order bound of the stable one."""
    rng = np.random.default_rng(31)
    ps = synth.two_species_set(40000, 15000, 17, grid=32).with_brightness([0.05, 0.3])
    # a crowded spot: its tiles are split over several work items
    k = 20000
    ps.x[:k] = 0.5 + rng.normal(0, 0.002, k)
    ps.y[:k] = 0.5 + rng.normal(0, 0.002, k)
    sc = render.Scene(ps, "f32")
    cam = synth.front_camera(200, 150)
    first = sc.render(cam, render.RenderParams(tile=T, accum=True, stable=True)).clone()
    other = render.Scene(synth.plain_set(5000, 3), "f32")
    other.render(synth.front_camera(64, 64))
    for bp in (0, 4096, 30000):
        again = sc.render(cam, render.RenderParams(tile=T, accum=True, stable=True, block_particles=bp))
        assert torch.equal(first, again), (T, bp)
    n = _max_contributions(ps, cam)
    fast = sc.render(cam, render.RenderParams(tile=T, accum=True))
    assert torch.allclose(fast, first, rtol=(2 * (n - 1) + 2) * U32, atol=0.0), (T, n)


def test_stable_plan_replays_are_bitwise_equal_and_match_single_views():
    """A multi-view plan with stable tile lists replays (CUDA graph) to the same bits, and
    each view matches the view rendered alone within the summation-order bound (the plan
    cuts its lists into work items for all views at once, so slice boundaries differ)."""
    ps = synth.two_species_set(30000, 10000, 41, grid=32).with_brightness([0.05, 0.3])
    cams = synth.orbit_cameras(5, 128, 96)
    sc = render.Scene(ps, "f32")
    plan = render.Plan(sc, cams, render.RenderParams(accum=True, stable=True), graph=True)
    out = plan.new_output()
    plan.launch(out)
    plan.check()
    first = out.clone()
    for _ in range(2):
        plan.launch(out)
        plan.check()
        assert torch.equal(out, first)
    for v, cam in enumerate(cams):
        alone = sc.render(cam, render.RenderParams(accum=True, stable=True))
        n = _max_contributions(ps, cam)
        assert torch.allclose(first[v], alone, rtol=(2 * (n - 1) + 2) * U32, atol=0.0), v


def test_plan_per_view_brightness_matches_rescaled_scenes():
    """A brightness sequence over the views of one plan (replayed as a CUDA graph) renders
    what separate scenes with the scaled brightness render; None restores the scales."""
    ps = synth.two_species_set(30000, 10000, 13, grid=32).with_brightness([0.05, 0.3])
    cams = synth.orbit_cameras(3, 128, 96)
    scale = np.array([[1.0, 1.0], [0.25, 2.0], [0.0, 0.7]], np.float32)
    sc = render.Scene(ps, "f32")
    plan = render.Plan(sc, cams, render.RenderParams(), graph=True)
    out = plan.new_output()
    plan.launch(out)
    plain = out.clone()
    plan.set_brightness(scale)
    plan.launch(out)
    plan.check()
    for v, cam in enumerate(cams):
        want = render.Scene(ps.with_brightness(ps.brightness * scale[v]), "f32").render(cam)
        assert torch.abs(out[v] - want).max().item() <= 1e-4, v
    plan.set_brightness(None)
    plan.launch(out)
    plan.check()
    assert torch.abs(out - plain).max().item() <= 1e-6
    with pytest.raises(_lib.SplotchError):
        plan.set_brightness(np.full((3, 2), -1.0, np.float32))
    plan.close()


def _thresholded(cmap, lo, hi):
    """Palette thresholds as a colormap: below lo and above hi the end colours repeat
    (resampled to 512 entries)."""
    t = np.linspace(0.0, 1.0, 512)
    u = np.clip((t - lo) / (hi - lo), 0.0, 1.0) * (cmap.shape[0] - 1)
    k = np.minimum(u.astype(np.int64), cmap.shape[0] - 2)
    f = (u - k)[:, None]
    return ((1.0 - f) * cmap[k] + f * cmap[k + 1]).astype(np.float32)


def test_plan_per_view_colormaps_match_the_oracle():
    """A colormap sequence over the views of one plan (graph replays), alone and with a
    brightness sequence, against the FP64 oracle rendering each view with that view's
    colormaps; None restores the scene's; a vector-colour scene refuses it."""
    import oracle
    ps = synth.two_species_set(30000, 10000, 17, grid=32).with_brightness([0.05, 0.3])
    cams = synth.orbit_cameras(3, 128, 96)
    rng = np.random.default_rng(3)
    maps = [[synth.smooth_ramp_cmap(rng, n=int(rng.integers(2, 300))) for _ in range(2)] for _ in range(3)]
    maps[1][0] = _thresholded(ps.cmaps[0], 0.2, 0.6)  # palette thresholds on the gas
    sc = render.Scene(ps, "f32")
    plan = render.Plan(sc, cams, render.RenderParams(tile=16), graph=True)
    out = plan.new_output()
    plan.launch(out)
    plain = out.clone()

    def check(scale):
        for v, cam in enumerate(cams):
            pv = ps.with_brightness(ps.brightness * (1.0 if scale is None else scale[v]))
            pv.cmaps = maps[v]
            want = oracle.final(oracle.render(pv, cam))
            assert np.abs(out[v].cpu().numpy() - want).max() <= 1e-4, v

    plan.set_colormaps(maps)
    plan.launch(out)
    plan.launch(out)
    plan.check()
    check(None)
    scale = np.array([[1.0, 0.5], [2.0, 1.0], [0.3, 3.0]], np.float32)
    plan.set_brightness(scale)
    plan.launch(out)
    plan.check()
    check(scale)
    # larger maps move the plan's colormap storage: the graph is captured again
    maps = [[synth.smooth_ramp_cmap(rng, n=4096) for _ in range(2)] for _ in range(3)]
    plan.set_colormaps(maps)
    plan.launch(out)
    plan.check()
    check(scale)
    plan.set_brightness(None)
    plan.set_colormaps(None)
    plan.launch(out)
    plan.check()
    assert torch.abs(out - plain).max().item() <= 1e-6
    with pytest.raises(_lib.SplotchError) as e:
        plan.set_colormaps([[np.full((3, 3), np.nan, np.float32)] * 2] * 3)
    assert e.value.status == _lib.INVALID_ARG
    plan.close()
    sc.close()
    vec = synth.with_vector_colour(ps, [1], 1)
    sv = render.Scene(vec, "f32")
    pv = render.Plan(sv, cams, render.RenderParams(tile=16))
    with pytest.raises(_lib.SplotchError) as e:
        pv.set_colormaps(maps)
    assert e.value.status == _lib.UNSUPPORTED
    pv.close()
    sv.close()


def test_plan_per_view_colormaps_with_cta_tiles():
    """Per-view colormaps through the CTA kernel (tiles above 32 px read the view's table
    at run time), against the oracle per view."""
    import oracle
    ps = synth.two_species_set(20000, 8000, 19, grid=32).with_brightness([0.05, 0.3])
    cams = synth.orbit_cameras(2, 120, 100)
    rng = np.random.default_rng(4)
    maps = [[synth.smooth_ramp_cmap(rng, n=int(rng.integers(2, 100))) for _ in range(2)] for _ in range(2)]
    sc = render.Scene(ps, "f32")
    plan = render.Plan(sc, cams, render.RenderParams(tile=40))
    plan.set_colormaps(maps)
    out = plan.new_output()
    plan.launch(out)
    plan.check()
    for v, cam in enumerate(cams):
        pv = ps.with_brightness(ps.brightness)
        pv.cmaps = maps[v]
        assert np.abs(out[v].cpu().numpy() - oracle.final(oracle.render(pv, cam))).max() <= 1e-4, v
    plan.close()
    sc.close()


@pytest.mark.parametrize("tile", [16, 40])
def test_far_plane_matches_the_oracle(tile):
    """A camera with a far plane culls the particles beyond it in the additive path (warp
    and CTA kernels), as the oracle's FP32 rule does."""
    import oracle
    ps = synth.two_species_set(30000, 10000, 23, grid=32).with_brightness([0.05, 0.3])
    cam = synth.front_camera(130, 100)
    cam.z_far = 2.1
    ref = oracle.final(oracle.render(ps, cam))
    got = render.Scene(ps, "f32").render(cam, render.RenderParams(tile=tile)).cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-4
    full = oracle.final(oracle.render(ps, synth.front_camera(130, 100)))
    assert np.abs(full - ref).max() > 1e-2  # the plane cut something
