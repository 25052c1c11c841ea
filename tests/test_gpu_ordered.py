"""Depth-ordered rendering (absorption different from emission) on the GPU: the radix
sort that orders the tile lists, and the ordered render against the FP64 oracle (needs a
GB300)."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1606_04427_gb300 import _lib, build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    assert torch.cuda.is_available()


def _sorted_on_gpu(keys, vals, lo, hi):
    wide = keys.dtype == np.uint64
    k = torch.from_numpy(keys.view(np.int64 if wide else np.int32)).cuda()
    v = torch.from_numpy(vals.view(np.int32)).cuda()
    _lib.check(_lib.load().splotch_debug_sort(k.data_ptr(), 8 if wide else 4, v.data_ptr(), keys.shape[0], lo, hi,
                                              None), "debug_sort")
    return k.cpu().numpy().view(keys.dtype), v.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("n", [2, 7, 4096, 4097, 12289, 1_000_003])
def test_radix_sort_is_a_stable_sort_by_the_chosen_bits(n):
    """Sorting by key bits [lo, hi) must equal a stable sort by those bits (numpy), so
    equal keys keep their input order; many equal digits and equal keys are included."""
    rng = np.random.default_rng(n)
    tile = rng.integers(0, 300, n).astype(np.uint64)
    depth = rng.integers(0, 1 << 32, n, dtype=np.uint64)
    depth[rng.random(n) < 0.3] = 12345  # runs of equal depth keys
    keys = (tile << np.uint64(32)) | depth
    vals = np.arange(n, dtype=np.uint32)
    for lo, hi in ((0, 32), (32, 48), (0, 64), (8, 16)):
        mask = np.uint64(((1 << (hi - lo)) - 1) << lo) if hi - lo < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
        order = np.argsort(keys & mask, kind="stable")
        k, v = _sorted_on_gpu(keys.copy(), vals.copy(), lo, hi)
        assert np.array_equal(k, keys[order]), (lo, hi)
        assert np.array_equal(v, vals[order]), (lo, hi)
    # depth bits then tile bits, each pass stable: tile-major, depth-minor order
    k1, v1 = _sorted_on_gpu(keys.copy(), vals.copy(), 0, 32)
    k2, v2 = _sorted_on_gpu(k1, v1, 32, 48)
    order = np.lexsort((vals, depth, tile))
    assert np.array_equal(v2, vals[order])


@pytest.mark.parametrize("n", [3, 4096, 100_003])
def test_radix_sort_with_32_bit_keys(n):
    """The 32-bit-key form the depth-ordered binning uses (particle depth keys, then tile
    ids): equal to numpy's stable sort by the chosen bits, with ties and an all-ones key."""
    rng = np.random.default_rng(7 + n)
    keys = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    keys[rng.random(n) < 0.25] = 0x7F00FF00
    keys[rng.random(n) < 0.1] = 0xFFFFFFFF
    vals = np.arange(n, dtype=np.uint32)
    for lo, hi in ((0, 32), (0, 16), (8, 24), (24, 32)):
        mask = np.uint32(((1 << (hi - lo)) - 1) << lo)
        order = np.argsort(keys & mask, kind="stable")
        k, v = _sorted_on_gpu(keys.copy(), vals.copy(), lo, hi)
        assert np.array_equal(k, keys[order]), (lo, hi)
        assert np.array_equal(v, vals[order]), (lo, hi)


import oracle  # noqa: E402
from paper_1606_04427_gb300 import render, synth  # noqa: E402

TOL_O = {"f32": 1e-4, "f16": 2e-3}


def _species_set(seed, n_gas=40000, n_star=15000):
    return synth.two_species_set(n_gas, n_star, seed, grid=64).with_brightness([0.05, 0.3])


def test_ordered_with_unit_absorption_is_the_standard_image():
    """Absorption = emission for every species: the ordered transfer telescopes to
    1 - exp(-a), the image of the additive path."""
    ps = _species_set(21)
    cam = synth.front_camera(192, 160)
    sc = render.Scene(ps, "f32")
    std = sc.render(cam).cpu().numpy()
    got = sc.render_ordered(cam, [1.0, 1.0]).cpu().numpy()
    assert np.abs(got - std).max() <= 1e-4
    # a common factor s: (1 - exp(-s a)) / s
    a = sc.render(cam, render.RenderParams(accum=True)).cpu().numpy().astype(np.float64)
    got = sc.render_ordered(cam, [2.5, 2.5]).cpu().numpy()
    assert np.abs(got - (1.0 - np.exp(-2.5 * a)) / 2.5).max() <= 1e-4


@pytest.mark.parametrize("tile", [8, 16, 24, 32])
def test_ordered_matches_the_depth_ordered_oracle(tile):
    """Species with different absorption (order matters): against the oracle's transfer
    applied farthest first, for tiles rendered whole and as four squares."""
    ps = _species_set(22 + tile)
    cam = synth.front_camera(200, 150)
    absorb = [2.0, 0.3]
    ref = oracle.render_rt_depth(ps, cam, absorb)
    got = render.Scene(ps, "f32").render_ordered(cam, absorb, render.RenderParams(tile=tile)).cpu().numpy()
    err = float(np.abs(got - ref).max())
    assert err <= TOL_O["f32"], (tile, err)
    # the order matters for this scene: the additive closed form is far off
    assert np.abs(ref - oracle.final(oracle.render(ps, cam))).max() > 1e-2


@pytest.mark.parametrize("absorb", [[0.1, 0.02], [2.0, 0.3], [8.0, 3.0]])
def test_ordered_each_transfer_path_matches_the_oracle(absorb):
    """The splat picks, per record, the degree-2 series (largest x = s E below 0.015), the
    degree-5 series (up to 0.25) or the exponential; these absorptions put the records of
    the scene (emission up to 0.05 and 0.3) on each path in turn."""
    ps = _species_set(44)
    cam = synth.front_camera(176, 144)
    ref = oracle.render_rt_depth(ps, cam, absorb)
    got = render.Scene(ps, "f32").render_ordered(cam, absorb, render.RenderParams(tile=16)).cpu().numpy()
    err = float(np.abs(got - ref).max())
    assert err <= TOL_O["f32"], (absorb, err)


def test_ordered_split_tiles_compose_their_slices():
    """A crowded tile is cut into slices of the depth-sorted list; the slices' affine maps
    compose far to near.  Also zero absorption (additive species) and FP16 storage."""
    rng = np.random.default_rng(5)
    n = 60000
    x = 0.5 + 0.01 * rng.standard_normal(n)
    y = 0.5 + 0.01 * rng.standard_normal(n)
    z = rng.uniform(0.2, 0.8, n)
    h = np.exp(rng.uniform(np.log(0.002), np.log(0.02), n))
    import oracle_pins as P
    cm = np.array([[0.2, 0.5, 0.9], [0.9, 0.4, 0.1]], np.float32)
    ps = P.make_set(x, y, z, h, rng.uniform(0, 1, n), type_begin=[0, n // 2, n], cmaps=[cm, cm[::-1].copy()],
                    betas=[0.02, 0.05])
    cam = synth.front_camera(96, 96)
    for absorb, storage in (([1.5, 0.0], "f32"), ([0.7, 3.0], "f16")):
        sc = render.Scene(ps, storage)
        assert sc.debug_bins(cam, render.RenderParams(tile=16))[0].max() > 4096  # split tiles
        ref = oracle.render_rt_depth(ps, cam, absorb, storage=storage)
        got = sc.render_ordered(cam, absorb, render.RenderParams(tile=16)).cpu().numpy()
        assert np.abs(got - ref).max() <= TOL_O[storage], (absorb, storage)


@pytest.mark.parametrize("tile", [16, 32])
def test_ordered_equal_depths_apply_in_index_order(tile):
    """Particles on three planes of equal depth, the species mixed on each plane: equal
    depths must be applied in particle-index order, as the oracle does, not in the order
    the binning's atomics happen to store them."""
    import oracle_pins as P
    rng = np.random.default_rng(40 + tile)
    n = 30000
    z = rng.choice(np.array([0.35, 0.5, 0.65], np.float32), n)
    cm = np.array([[0.2, 0.5, 0.9], [0.9, 0.4, 0.1]], np.float32)
    ps = P.make_set(rng.uniform(0.25, 0.75, n), rng.uniform(0.25, 0.75, n), z,
                    np.exp(rng.uniform(np.log(0.004), np.log(0.03), n)), rng.uniform(0, 1, n),
                    type_begin=[0, n // 2, n], cmaps=[cm, cm[::-1].copy()], betas=[0.05, 0.1])
    cam = synth.front_camera(160, 128)
    r = oracle.raster(ps, cam)
    zc = r["zc"][r["active"]]
    assert np.unique(zc).shape[0] < zc.shape[0] // 100  # nearly every depth is shared
    absorb = [2.5, 0.2]
    ref = oracle.render_rt_depth(ps, cam, absorb)
    got = render.Scene(ps, "f32").render_ordered(cam, absorb, render.RenderParams(tile=tile)).cpu().numpy()
    assert np.abs(got - ref).max() <= TOL_O["f32"]


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_ordered_reduced_precision_storage(storage):
    """The ordered render of a scene stored in BF16 / FP16, against the oracle fed the same
    rounded attributes (bar 2e-3)."""
    ps = _species_set(50)
    cam = synth.front_camera(150, 120)
    absorb = [2.0, 0.3]
    ref = oracle.render_rt_depth(ps, cam, absorb, storage=storage)
    got = render.Scene(ps, storage).render_ordered(cam, absorb, render.RenderParams(tile=24)).cpu().numpy()
    assert np.abs(got - ref).max() <= 2e-3, storage


def test_ordered_degenerate_scenes():
    """No particles, every particle behind the camera, and a single particle: the ordered
    render writes a black image, or the one particle's closed form (I = (E/A)(1 - e^-A w)
    per pixel, from the oracle), over the whole (ragged) image."""
    import oracle_pins as P
    cam = synth.front_camera(77, 53)
    absorb = [1.3]
    empty = P.make_set(np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0))
    out = torch.full((53, 77, 3), float("nan"), device="cuda")
    got = render.Scene(empty, "f32").render_ordered(cam, absorb, out=out).cpu().numpy()
    assert np.array_equal(got, np.zeros_like(got))
    behind = P.make_set([0.5] * 50, [0.5] * 50, np.linspace(3.0, 4.0, 50), [0.01] * 50)
    out.fill_(float("nan"))
    got = render.Scene(behind, "f32").render_ordered(cam, absorb, out=out).cpu().numpy()
    assert np.array_equal(got, np.zeros_like(got))
    one = P.make_set([0.5], [0.52], [0.5], [0.02], [0.7], beta=0.4)
    ref = oracle.render_rt_depth(one, cam, absorb)
    got = render.Scene(one, "f32").render_ordered(cam, absorb, render.RenderParams(tile=8)).cpu().numpy()
    assert ref.max() > 0.05 and np.abs(got - ref).max() <= 1e-5


def test_ordered_one_crowded_tile_many_slices():
    """Forty thousand particles on one tile: its list is cut into many slices whose maps
    compose far to near; also the tile of 32 px rendered as four squares."""
    import oracle_pins as P
    rng = np.random.default_rng(8)
    n = 40000
    cm = np.array([[0.2, 0.5, 0.9], [0.9, 0.4, 0.1]], np.float32)
    ps = P.make_set(0.5 + 0.002 * rng.standard_normal(n), 0.5 + 0.002 * rng.standard_normal(n),
                    rng.uniform(0.3, 0.7, n), np.full(n, 0.001), rng.uniform(0, 1, n),
                    type_begin=[0, n // 2, n], cmaps=[cm, cm[::-1].copy()], betas=[0.01, 0.02])
    cam = synth.front_camera(70, 70)
    absorb = [3.0, 0.5]
    ref = oracle.render_rt_depth(ps, cam, absorb)
    for tile in (16, 32):
        got = render.Scene(ps, "f32").render_ordered(cam, absorb, render.RenderParams(tile=tile)).cpu().numpy()
        assert np.abs(got - ref).max() <= TOL_O["f32"], tile


@pytest.mark.parametrize("tile", [16, 32])
def test_ordered_map_output_matches_the_oracle_map(tile):
    """SPLOTCH_OUT_MAP: per pixel the affine map (alpha, beta) of the ordered transfer,
    against the oracle's, on a scene with split tiles (their slices' alphas multiply)."""
    import oracle_pins as P
    rng = np.random.default_rng(12)
    n = 30000
    cm = np.array([[0.2, 0.5, 0.9], [0.9, 0.4, 0.1]], np.float32)
    x = np.concatenate([0.5 + 0.004 * rng.standard_normal(n // 2), rng.uniform(0.3, 0.7, n - n // 2)])
    y = np.concatenate([0.5 + 0.004 * rng.standard_normal(n // 2), rng.uniform(0.3, 0.7, n - n // 2)])
    ps = P.make_set(x, y, rng.uniform(0.3, 0.7, n), np.exp(rng.uniform(np.log(0.002), np.log(0.02), n)),
                    rng.uniform(0, 1, n), type_begin=[0, n // 3, n], cmaps=[cm, cm[::-1].copy()], betas=[0.03, 0.1])
    cam = synth.front_camera(110, 90)
    absorb = [3.0, 0.5]
    A, B = oracle.render_rt_depth_map(ps, cam, absorb)
    sc = render.Scene(ps, "f32")
    assert sc.debug_bins(cam, render.RenderParams(tile=tile))[0].max() > 4096  # split tiles
    got = sc.render_ordered(cam, absorb, render.RenderParams(tile=tile, map=True)).cpu().numpy()
    assert got.shape == (90, 110, 6)
    assert np.abs(got[..., :3] - A).max() <= 1e-4 and np.abs(got[..., 3:] - B).max() <= 1e-4
    assert A.min() < 0.5  # the maps really absorb


def test_depth_slab_maps_compose_on_the_gpu():
    """Three depth slabs (cameras with near / far planes) rendered as maps on the GPU and
    composed far to near equal the whole ordered frame."""
    from paper_1606_04427_gb300 import shard
    ps = _species_set(61)
    cam = synth.front_camera(160, 120)
    absorb = [2.0, 0.3]
    sc = render.Scene(ps, "f32")
    whole = sc.render_ordered(cam, absorb, render.RenderParams(tile=16))
    bounds = shard.slab_bounds(cam.z_near, 1.7, 2.3, 3)
    maps = [sc.render_ordered(shard.slab_camera(cam, bounds, k), absorb, render.RenderParams(tile=16, map=True))
            for k in range(3)]
    got = shard.compose_maps(list(reversed(maps)))[..., 3:]
    assert torch.abs(got - whole).max().item() <= 2e-5
    ref = oracle.render_rt_depth(ps, cam, absorb)
    assert np.abs(got.cpu().numpy() - ref).max() <= TOL_O["f32"]


def test_compose_maps_entry_point_against_the_oracle():
    """splotch_compose_maps against the oracle's FP64 composition: the oracle's own slab
    maps (three depth slabs) composed far to near on the GPU equal the oracle's whole
    frame; random maps of 1, 2 and 5 slabs with a ragged pixel count agree with the
    oracle's composition of the same FP32 inputs; bad arguments are rejected."""
    from paper_1606_04427_gb300 import shard
    ps = _species_set(62)
    cam = synth.front_camera(97, 53)
    absorb = [2.0, 0.3]
    bounds = shard.slab_bounds(cam.z_near, 1.7, 2.3, 3)
    slabs = []
    for k in range(3):
        A, B = oracle.render_rt_depth_map(ps, shard.slab_camera(cam, bounds, k), absorb)
        slabs.append(np.concatenate([A, B], -1).astype(np.float32))
    far_to_near = slabs[::-1]
    got = shard.compose_maps([torch.from_numpy(m).cuda() for m in far_to_near]).cpu().numpy()
    want = oracle.compose_maps(far_to_near)
    assert np.abs(got - want).max() <= 2e-6 * max(1.0, np.abs(want).max())
    whole = oracle.render_rt_depth(ps, cam, absorb)
    assert np.abs(got[..., 3:] - whole).max() <= TOL_O["f32"]
    rng = np.random.default_rng(63)
    for n in (1, 2, 5):
        ms = [np.concatenate([rng.uniform(0, 1, (7, 13, 3)), rng.uniform(0, 2, (7, 13, 3))], -1).astype(np.float32)
              for _ in range(n)]
        got = shard.compose_maps([torch.from_numpy(m).cuda() for m in ms]).cpu().numpy()
        want = oracle.compose_maps(ms)
        assert np.abs(got - want).max() <= 1e-5 * max(1.0, np.abs(want).max()), n
    lib = _lib.load()
    buf = torch.zeros(2 * 6 * 10, device="cuda")
    assert lib.splotch_compose_maps(buf.data_ptr(), 0, 10, buf.data_ptr(), None) == _lib.INVALID_ARG
    assert lib.splotch_compose_maps(buf.data_ptr(), 2, 10, buf.data_ptr(), None) == _lib.INVALID_ARG  # overlap
    assert lib.splotch_compose_maps(None, 1, 10, buf.data_ptr(), None) == _lib.INVALID_ARG


def test_ordered_rejects_large_tiles_and_bad_absorption():
    sc = render.Scene(_species_set(30, 2000, 500), "f32")
    cam = synth.front_camera(128, 128)
    with pytest.raises(_lib.SplotchError) as e:
        sc.render_ordered(cam, [1.0, 1.0], render.RenderParams(tile=40))
    assert e.value.status == _lib.UNSUPPORTED
    with pytest.raises(_lib.SplotchError) as e:
        sc.render_ordered(cam, [1.0, -1.0])
    assert e.value.status == _lib.INVALID_ARG
