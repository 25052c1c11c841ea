"""CUDA path against the FP64 CPU oracle through the C ABI (needs a GB300).

Bars (stated per result in the assertion messages):
  * raster decisions (X, Y, R, z_c, active) and tile binning (counts, offsets,
    member sets) are bit-exact: both sides evaluate the documented FP32 rule;
  * images: max absolute per-channel error on O = 1 - exp(-a) <= 1e-4 for FP32
    storage and <= 2e-3 for FP16 / BF16 storage (oracle fed the same rounded
    attributes); the accumulation a is also gated relatively (FP32: 2e-5), so
    saturation of O cannot hide an error.
"""
import numpy as np
import pytest
import torch

import oracle
import oracle_pins as P
from paper_1606_04427_gb300 import _lib, build, render, synth

pytestmark = pytest.mark.gpu

TOL_O = {"f32": 1e-4, "f16": 2e-3, "bf16": 2e-3}
RTOL_A_F32 = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    assert torch.cuda.is_available()
    _lib.load()


def _sets():
    return {
        "plain": (synth.plain_set(20000, 0), synth.front_camera(256, 256)),
        "clustered": (synth.clustered_set(60000, 1, grid=64).with_brightness([0.05]),
                      synth.front_camera(200, 130)),
        "two_species": (synth.two_species_set(40000, 15000, 2, grid=64).with_brightness([0.05, 0.3]),
                        synth.front_camera(192, 160)),
        "tiny": P.tiny_scene(3, n=64, W=40, H=28),
    }


SETS = _sets()


def _compare_image(name, ps, cam, storage, params=None, scene=None):
    params = params or render.RenderParams()
    sc = scene or render.Scene(ps, storage)
    a_g = sc.render(cam, render.RenderParams(**{**params.__dict__, "accum": True})).cpu().numpy().astype(np.float64)
    O_g = sc.render(cam, params).cpu().numpy().astype(np.float64)
    op = oracle.Params(tile=params.tile or 32, rfac=params.rfac, sigma_over_R=params.sigma_over_R,
                       r_min_px=params.r_min_px)
    a_o = oracle.render(ps, cam, op, storage)
    O_o = oracle.final(a_o)
    errO = np.abs(O_g - O_o).max()
    scale = np.abs(a_o) + 1e-6 * max(1e-30, np.abs(a_o).max())
    rel_a = (np.abs(a_g - a_o) / scale).max()
    assert errO <= TOL_O[storage], f"{name}/{storage}: max |dO| = {errO:.3e} > {TOL_O[storage]}"
    if storage == "f32":
        assert rel_a <= RTOL_A_F32, f"{name}: max rel |da| = {rel_a:.3e}"
    assert np.abs(a_o).max() > 0 or name == "empty"
    return errO, rel_a


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("name", sorted(SETS))
def test_raster_bitexact(name, storage):
    ps, cam = SETS[name]
    sc = render.Scene(ps, storage)
    g = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in sc.debug_raster(cam).items()}
    o = oracle.raster(ps, cam, storage=storage)
    assert np.array_equal(g["active"], o["active"]), f"{name}/{storage}: active flags differ"
    assert np.array_equal(g["zc"].view(np.uint32), o["zc"].astype(np.float32).view(np.uint32))
    a = o["active"]
    for k in ("X", "Y", "R"):
        assert np.array_equal(g[k][a].view(np.uint32), o[k][a].astype(np.float32).view(np.uint32)), (name, k)
    err = np.abs(g["e"][a] - o["e"][a]).max() if a.any() else 0.0
    emax = np.abs(o["e"]).max()
    bound = 2e-6 * emax if storage == "f32" else 2e-3 * emax
    assert err <= bound, f"{name}/{storage}: colour error {err:.3e} > {bound:.3e}"


@pytest.mark.parametrize("T", [8, 16, 24, 32, 64])
@pytest.mark.parametrize("name", sorted(SETS))
def test_binning_bitexact(name, T):
    ps, cam = SETS[name]
    sc = render.Scene(ps, "f32")
    c_g, o_g, m_g = sc.debug_bins(cam, render.RenderParams(tile=T))
    c_o, o_o, m_o = oracle.bins(ps, cam, oracle.Params(tile=T))
    assert np.array_equal(c_g, c_o), f"{name}/T={T}: counts differ"
    assert np.array_equal(o_g, o_o), f"{name}/T={T}: offsets differ"
    assert np.array_equal(m_g, m_o), f"{name}/T={T}: member lists differ"


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("name", sorted(SETS))
def test_image_parity(name, storage):
    ps, cam = SETS[name]
    _compare_image(name, ps, cam, storage)


def test_config0_full_size():
    """Plain single view, FP32: 100k particles, 256^2, full image against the oracle."""
    ps = synth.plain_set(100_000, 0).with_brightness([0.25])
    _compare_image("plain100k", ps, synth.front_camera(256, 256), "f32")


@pytest.mark.parametrize("T", [8, 16, 24, 40, 48, 64])
def test_tile_size_invariance(T):
    ps, cam = SETS["clustered"]
    sc = render.Scene(ps, "f32")
    base = sc.render(cam, render.RenderParams(tile=32)).cpu().numpy()
    other = sc.render(cam, render.RenderParams(tile=T)).cpu().numpy()
    assert np.abs(base - other).max() <= 1e-4


def test_ragged_and_tiny_images():
    ps = synth.plain_set(5003, 4)
    for (W, H, T) in [(1, 1, 8), (1, 300, 16), (300, 1, 16), (37, 23, 8), (129, 65, 64), (100, 70, 3)]:
        cam = synth.front_camera(W, H)
        _compare_image(f"{W}x{H}/T{T}", ps, cam, "f32", render.RenderParams(tile=T))


def test_empty_and_all_culled():
    ps = synth.plain_set(1000, 5)
    sc = render.Scene(ps, "f32")
    away = synth.Camera((0.5, 0.5, -1.5), (0.5, 0.5, -3.0), (0, 1, 0), 45.0, 1e-3, 64, 48)
    img = sc.render(away).cpu().numpy()
    assert img.shape == (48, 64, 3) and np.all(img == 0.0)
    empty = P.make_set(np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0))
    sc0 = render.Scene(empty, "f32")
    img = sc0.render(synth.front_camera(33, 17)).cpu().numpy()
    assert np.all(img == 0.0)


def test_crowded_tile_is_split_and_merged():
    """Twenty thousand particles on one spot: the tile holds far more than one work
    item's share, so it is cut into slices whose partial sums merge in scratch."""
    rng = np.random.default_rng(9)
    n = 20000
    x = 0.5 + rng.normal(0, 0.004, n)
    y = 0.5 + rng.normal(0, 0.004, n)
    z = 0.5 + rng.normal(0, 0.004, n)
    ps = P.make_set(x, y, z, np.full(n, 0.004), rng.uniform(0, 1, n), beta=0.01)
    cam = synth.front_camera(96, 96)
    for T in (16, 32, 64):
        _compare_image(f"crowded/T{T}", ps, cam, "f32", render.RenderParams(tile=T))


def test_large_particles_cover_many_tiles():
    """Particles close to the camera cover most of the image: they stay on the GPU and
    are rendered by every tile they touch."""
    rng = np.random.default_rng(10)
    n = 300
    ps = P.make_set(rng.uniform(0.3, 0.7, n), rng.uniform(0.3, 0.7, n), rng.uniform(2.2, 2.45, n),
                    rng.uniform(0.01, 0.05, n), rng.uniform(0, 1, n), beta=0.02)
    cam = synth.front_camera(160, 120)
    _compare_image("large", ps, cam, "f32", render.RenderParams(tile=16))


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_mid_size_ragged_image_with_mixed_particles(storage):
    """A ragged 1000 x 760 image at 16-px tiles (63 x 48 tiles, the last row and column
    partial) with small particles, particles across tile edges, a crowded spot (split
    tiles) and large particles near the camera (binned by whole warps), against the
    oracle."""
    rng = np.random.default_rng(21)
    n1, n2, n3 = 120000, 20000, 150
    x = np.concatenate([rng.uniform(0.0, 1.0, n1), 0.5 + rng.normal(0, 0.01, n2), rng.uniform(0.3, 0.7, n3)])
    y = np.concatenate([rng.uniform(0.0, 1.0, n1), 0.45 + rng.normal(0, 0.01, n2), rng.uniform(0.3, 0.7, n3)])
    z = np.concatenate([rng.uniform(0.0, 1.0, n1), 0.5 + rng.normal(0, 0.01, n2), rng.uniform(1.6, 2.2, n3)])
    h = np.concatenate([rng.uniform(0.0005, 0.006, n1), np.full(n2, 0.002), rng.uniform(0.005, 0.02, n3)])
    ps = P.make_set(x, y, z, h, rng.uniform(0, 1, n1 + n2 + n3), beta=0.01)
    _compare_image("mid_size", ps, synth.front_camera(1000, 760), storage, render.RenderParams(tile=16))


def test_multi_view_render_matches_single_views():
    ps, _ = SETS["clustered"]
    cams = synth.orbit_cameras(5, 120, 90)
    sc = render.Scene(ps, "f32")
    multi = sc.render(cams).cpu().numpy()
    for v, cam in enumerate(cams):
        single = sc.render(cam).cpu().numpy()
        assert np.abs(multi[v] - single).max() <= 1e-4
        O_o = oracle.final(oracle.render(ps, cam))
        assert np.abs(multi[v] - O_o).max() <= 1e-4


@pytest.mark.parametrize("graph", [False, True])
def test_plan_matches_single_views(graph):
    ps, _ = SETS["two_species"]
    cams = synth.orbit_cameras(8, 96, 96)
    sc = render.Scene(ps, "f16")
    plan = render.Plan(sc, cams, render.RenderParams(tile=16), headroom=1.3, graph=graph)
    out = plan.new_output()
    for _ in range(3):
        plan.launch(out)
        plan.check()
        got = out.cpu().numpy()
        for v, cam in enumerate(cams):
            single = sc.render(cam, render.RenderParams(tile=16)).cpu().numpy()
            assert np.abs(got[v] - single).max() <= 2e-4
            O_o = oracle.final(oracle.render(ps, cam, oracle.Params(tile=16), "f16"))
            assert np.abs(got[v] - O_o).max() <= TOL_O["f16"]
    plan.close()


def test_plan_reports_capacity_overflow():
    """A plan sized on cameras that see nothing cannot hold a frame that sees the data:
    its kernels skip the work and the check reports CAPACITY with the pairs needed."""
    ps, _ = SETS["plain"]
    sc = render.Scene(ps, "f32")
    away = [synth.Camera((0.5, 0.5, -1.5), (0.5, 0.5, -3.0), (0, 1, 0), 45.0, 1e-3, 64, 64)] * 2
    plan = render.Plan(sc, away, headroom=1.0, graph=True)
    out = plan.new_output()
    plan.launch(out)
    assert plan.check() == 0
    plan.set_cameras([synth.front_camera(64, 64)] * 2)
    plan.launch(out)
    with pytest.raises(_lib.SplotchError) as ei:
        plan.check()
    assert ei.value.status == _lib.CAPACITY
    plan.close()


def test_allocator_failure_reports_oom():
    ps = synth.plain_set(2000, 6)
    never = render.CallbackAllocator(lambda n, s: 0, lambda p, s: None)
    with pytest.raises(_lib.SplotchError) as ei:
        render.Scene(ps, "f32", allocator=never)
    assert ei.value.status == _lib.OOM
    # the scene fits (three allocations), the render workspace does not
    budget = {"n": 3}
    base = render.torch_allocator()

    def limited(n, s):
        if budget["n"] <= 0:
            return 0
        budget["n"] -= 1
        return base._alloc_py(n, s)

    alloc = render.CallbackAllocator(limited, base._free_py)
    sc = render.Scene(ps, "f32", allocator=alloc)
    with pytest.raises(_lib.SplotchError) as ei:
        sc.render(synth.front_camera(64, 64))
    assert ei.value.status == _lib.OOM
    budget["n"] = 100
    img = sc.render(synth.front_camera(64, 64)).cpu().numpy()
    assert img.max() > 0


def test_torch_allocator_path_matches_default():
    ps, cam = SETS["clustered"]
    a = render.Scene(ps, "f32").render(cam).cpu().numpy()
    b = render.Scene(ps, "f32", allocator=render.torch_allocator()).render(cam).cpu().numpy()
    assert np.abs(a - b).max() <= 1e-4


def test_bounded_wait_times_out_and_context_survives():
    lib = _lib.load()
    st = lib.splotch_selftest_bounded_wait(200_000, torch.cuda.current_stream().cuda_stream)
    assert st == _lib.TIMEOUT
    ps, cam = SETS["plain"]
    img = render.Scene(ps, "f32").render(cam, render.RenderParams(sync=True)).cpu().numpy()
    assert img.max() > 0


def test_device_inputs_match_host_inputs():
    ps, cam = SETS["two_species"]
    dev = synth.ParticleSet(**{k: getattr(ps, k) for k in ps.__dataclass_fields__})
    for k in ("x", "y", "z", "h", "intensity"):
        setattr(dev, k, torch.from_numpy(getattr(ps, k)).cuda())
    a = render.Scene(ps, "bf16").render(cam).cpu().numpy()
    b = render.Scene(dev, "bf16").render(cam).cpu().numpy()
    assert np.abs(a - b).max() <= 2e-4


def test_invalid_particles_rejected():
    ps = synth.plain_set(100, 7)
    ps.h[5] = 0.0
    with pytest.raises(_lib.SplotchError) as ei:
        render.Scene(ps, "f32")
    assert ei.value.status == _lib.INVALID_ARG
    ps = synth.plain_set(100, 7)
    ps.x[3] = np.nan
    with pytest.raises(_lib.SplotchError):
        render.Scene(ps, "f32")
