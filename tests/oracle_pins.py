"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each pin is a plain function that raises AssertionError when the oracle (the
build currently selected by ``oracle.using``, default the real one) is wrong.
``test_oracle_pins.py`` runs them on the real oracle; ``test_oracle_mutants.py``
runs them on copies of the oracle with planted mistakes and requires every
mistake to fail at least one pin.

None of these pins re-types the oracle's formulas: they check closed forms of
the pinhole camera and of the Gaussian integral, invariants (order, linearity,
tile-size independence), brute force on tiny scenes, the radiative-transfer
update the paper names, special cases of the colormap and normalisation, the
paper's tile-diagram example, and library routines for the storage codes.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

import oracle
from paper_1606_04427_gb300.synth import Camera, ParticleSet, TWO_POINT_CMAP, plain_set

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
C0 = (0.5, 0.5, 0.5)


def make_set(x, y, z, h, I=None, cmap=TWO_POINT_CMAP, beta=1.0, type_begin=None, cmaps=None,
             betas=None) -> ParticleSet:
    x = np.asarray(x, np.float32)
    n = x.shape[0]
    I = np.full(n, 0.5, np.float32) if I is None else np.asarray(I, np.float32)
    if type_begin is None:
        type_begin = [0, n]
    nt = len(type_begin) - 1
    cmaps = cmaps if cmaps is not None else [np.asarray(cmap, np.float32)] * nt
    betas = betas if betas is not None else [beta] * nt
    return ParticleSet(x, np.asarray(y, np.float32), np.asarray(z, np.float32),
                       np.asarray(h, np.float32), I, np.asarray(type_begin, np.int64), cmaps,
                       np.asarray(betas, np.float32), np.zeros(nt, np.int32),
                       np.zeros(nt, np.float32), np.ones(nt, np.float32))


def front(W, H, dist=2.0, fov=45.0, z_near=1e-3):
    return Camera((C0[0], C0[1], C0[2] + dist), C0, (0.0, 1.0, 0.0), fov, z_near, W, H)


def focal(H, fov=45.0):
    return (0.5 * H) / math.tan(math.radians(fov) / 2.0)


def world_for_screen(X, Y, W, H, depth=2.0, fov=45.0):
    """World point at ``depth`` in front of the +z front camera that a pinhole
    camera maps to pixel coordinates (X, Y): the textbook inverse projection."""
    F = focal(H, fov)
    return (C0[0] + (X - W / 2.0) * depth / F, C0[1] - (Y - H / 2.0) * depth / F,
            C0[2] + 2.0 - depth)


def tiny_scene(seed, n=48, W=32, H=24):
    """A few dozen particles around the view: some off-screen, some behind or at the
    camera, radii from sub-pixel to larger than the image."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-0.2, 1.2, n)
    y = rng.uniform(-0.2, 1.2, n)
    z = rng.uniform(-0.5, 1.5, n)
    z[:3] = [2.5, 2.7, 2.4995]        # at, behind, just in front of the camera plane
    h = np.exp(rng.uniform(np.log(0.002), np.log(0.3), n))
    I = rng.uniform(0.0, 1.0, n)
    return make_set(x, y, z, h, I), front(W, H, dist=2.0)


# ----------------------------------------------------------------------------------------
# camera and projection (Section 2.1)

def pin_lookat_projects_to_centre():
    ps = make_set([0.5], [0.5], [0.5], [0.01])
    for W, H in ((64, 64), (320, 200)):
        r = oracle.raster(ps, front(W, H))
        assert r["X"][0] == W / 2.0 and r["Y"][0] == H / 2.0, (r["X"][0], r["Y"][0])
    rng = np.random.default_rng(7)
    for _ in range(5):
        v = rng.standard_normal(3)
        v /= np.linalg.norm(v)
        cam = Camera(tuple(np.asarray(C0) + 1.7 * v), C0, (0.0, 1.0, 0.0), 45.0, 1e-3, 200, 120)
        r = oracle.raster(ps, cam)
        assert abs(r["X"][0] - 100.0) < 1e-3 and abs(r["Y"][0] - 60.0) < 1e-3


def pin_vertical_fov_edges():
    """A point at half the vertical field of view above the axis lands on the top
    edge, below on the bottom edge; horizontally the edge is at atan((W/2)/F)."""
    W, H, D = 320, 200, 2.0
    t = math.tan(math.radians(22.5))
    F = focal(H)
    pts = [(0.5, 0.5 + D * t, 0.5), (0.5, 0.5 - D * t, 0.5),
           (0.5 + D * (W / 2.0) / F, 0.5, 0.5), (0.5 - D * (W / 2.0) / F, 0.5, 0.5)]
    ps = make_set(*[[p[a] for p in pts] for a in range(3)], [0.001] * 4)
    r = oracle.raster(ps, front(W, H, dist=D))
    want = [(W / 2, 0.0), (W / 2, H), (W, H / 2), (0.0, H / 2)]
    for k, (wx, wy) in enumerate(want):
        assert abs(r["X"][k] - wx) < 2e-3 and abs(r["Y"][k] - wy) < 2e-3, (k, r["X"][k], r["Y"][k])


def pin_handedness():
    """Right-handed world, y up: from +z looking at the centre, +x is to the right;
    from +x looking at the centre, +z is to the left; +y is up (smaller row)."""
    c = np.asarray(C0)
    ps = make_set([0.8, 0.5, 0.5], [0.5, 0.8, 0.5], [0.5, 0.5, 0.8], [0.001] * 3)
    r = oracle.raster(ps, front(100, 100))
    assert r["X"][0] > 50 + 10 and abs(r["Y"][0] - 50) < 1e-3
    assert r["Y"][1] < 50 - 10 and abs(r["X"][1] - 50) < 1e-3
    side = Camera(tuple(c + [2.0, 0, 0]), C0, (0.0, 1.0, 0.0), 45.0, 1e-3, 100, 100)
    r = oracle.raster(ps, side)
    assert r["X"][2] < 50 - 10 and r["Y"][1] < 50 - 10


def pin_camera_rejections():
    bad = [Camera((0.5, 3.0, 0.5), C0, (0.0, 1.0, 0.0), 45.0, 1e-3, 8, 8),   # up along view
           Camera((0.5, 0.5, 2.5), C0, (0.0, 1.0, 0.0), 0.0, 1e-3, 8, 8),
           Camera((0.5, 0.5, 2.5), C0, (0.0, 1.0, 0.0), 180.0, 1e-3, 8, 8),
           Camera(C0, C0, (0.0, 1.0, 0.0), 45.0, 1e-3, 8, 8),
           Camera((0.5, 0.5, 2.5), C0, (0.0, 1.0, 0.0), 45.0, 0.0, 8, 8),
           Camera((0.5, 0.5, 2.5), C0, (0.0, 1.0, 0.0), 45.0, 1e-3, 0, 8)]
    for cam in bad:
        try:
            oracle.camera(cam)
        except ValueError:
            continue
        raise AssertionError(f"accepted {cam}")


def pin_projected_radius_is_projected_length():
    """r is the pinhole image of a length h at the particle's depth: two points a
    distance h apart across the view land r pixels apart."""
    W = H = 256
    hh = 0.05
    for depth in (1.0, 2.0, 3.5):
        z = C0[2] + 2.0 - depth
        ps = make_set([0.5, 0.5 + hh], [0.5, 0.5], [z, z], [hh, hh])
        r = oracle.raster(ps, front(W, H))
        sep = r["X"][1] - r["X"][0]
        assert abs(r["R"][0] - 0.75 * sep) < 1e-3 * sep, (depth, r["R"][0], sep)


def pin_radius_floor():
    ps = make_set([0.5, 0.5], [0.5, 0.5], [0.5, 0.5], [1e-6, 1e-4])
    r = oracle.raster(ps, front(64, 64))
    assert r["R"][0] == np.float32(0.75) and r["R"][1] == np.float32(0.75)


def pin_near_plane_cull():
    cam = front(64, 64, dist=2.0, z_near=0.01)
    # depths: behind, at camera, at the near plane (up to rounding), just beyond, far
    z = [2.6, 2.5, 2.49, 2.48, 0.5]
    ps = make_set([0.5] * 5, [0.5] * 5, z, [0.001] * 5)
    r = oracle.raster(ps, cam)
    assert list(r["active"]) == [False, False, r["zc"][2] > np.float32(0.01), True, True]
    assert not r["active"][0] and not r["active"][1] and r["active"][3]


def pin_far_plane_cull():
    """The far plane keeps z_c <= z_far (inclusive) and culls beyond; with no far plane
    (0 or infinite) nothing is culled for distance; z_far <= z_near is rejected."""
    z = [0.5, 0.49, 0.51, -3.0, 2.0]  # z_c = 2.5 - z: 2.0 exactly, 2.01, 1.99, 5.5, 0.5
    ps = make_set([0.5] * 5, [0.5] * 5, z, [0.001] * 5)
    cam = front(64, 64, dist=2.0)
    r = oracle.raster(ps, cam)
    assert r["zc"][0] == np.float32(2.0) and list(r["active"]) == [True] * 5
    cam.z_far = 2.0
    assert list(oracle.raster(ps, cam)["active"]) == [True, False, True, False, True]
    cam.z_far = float("inf")
    assert list(oracle.raster(ps, cam)["active"]) == [True] * 5
    cam.z_far = cam.z_near
    try:
        oracle.camera(cam)
        raise AssertionError("z_far <= z_near accepted")
    except ValueError:
        pass


def pin_depth_slabs_partition_the_particles():
    """Cameras that differ only in (z_near, z_far) = consecutive slab bounds make each
    active particle active in exactly one slab."""
    rng = np.random.default_rng(2)
    n = 5000
    ps = make_set(rng.uniform(0, 1, n), rng.uniform(0, 1, n), rng.uniform(0, 1, n), np.full(n, 0.004))
    bounds = [1e-3, 1.7, 2.0, 2.0001, 2.3, 0.0]
    seen = np.zeros(n, np.int64)
    for lo, hi in zip(bounds[:-1], bounds[1:]):
        cam = front(96, 96, dist=2.0, z_near=lo)
        cam.z_far = hi
        seen += oracle.raster(ps, cam)["active"]
    assert np.array_equal(seen, oracle.raster(ps, front(96, 96, dist=2.0))["active"].astype(np.int64))


# ----------------------------------------------------------------------------------------
# Gaussian footprint (Section 2.1) and additive drawing (Section 3.2.2)

def _single(R_px, W=160, H=160, X=None, Y=None, I=0.0, beta=1.0):
    X = W / 2.0 + 0.3 if X is None else X
    Y = H / 2.0 - 0.2 if Y is None else Y
    x, y, z = world_for_screen(X, Y, W, H)
    h = (R_px / 0.75) * 2.0 / focal(H)
    return make_set([x], [y], [z], [h], [I], beta=beta), front(W, H)


def pin_conservation():
    """Total deposit of one splat with sigma >= 16 px and its support inside the image
    equals the Gaussian integral over the disc d < R: e pi sigma^2 (1 - exp(-R^2/sigma^2))."""
    for R_px in (32.0, 45.5):
        ps, cam = _single(R_px)
        a = oracle.render(ps, cam)
        r = oracle.raster(ps, cam)
        e = r["e"][0]
        R = r["R"][0]
        sig = 0.5 * R
        want = math.pi * sig * sig * (1.0 - math.exp(-(R * R) / (sig * sig)))
        for c in range(3):
            got = a[:, :, c].sum() / e[c]
            assert abs(got / want - 1.0) < 1e-3, (R_px, c, got, want)


def pin_peak_and_cut():
    """A particle centred on a pixel centre deposits exactly its colour there; every
    deposit lies inside d < R and is at least e exp(-4) (sigma = R/2 cut at R)."""
    W = H = 64
    ps, cam = _single(6.0, W, H, X=32.5, Y=20.5)
    r = oracle.raster(ps, cam)
    a = oracle.render(ps, cam)
    e = r["e"][0]
    X, Y, R = r["X"][0], r["Y"][0], r["R"][0]
    assert abs(X - 32.5) < 1e-4 and abs(Y - 20.5) < 1e-4
    assert abs(a[20, 32, 0] - e[0]) < 1e-6 * e[0]
    jj, ii = np.nonzero(a[:, :, 0])
    d2 = (ii + 0.5 - X) ** 2 + (jj + 0.5 - Y) ** 2
    assert d2.max() < R * R * (1 + 1e-6)
    assert a[jj, ii, 0].min() >= e[0] * math.exp(-4.0) * (1 - 1e-6)
    # every pixel centre strictly inside 0.99 R got a deposit
    yy, xx = np.mgrid[0:H, 0:W]
    inside = ((xx + 0.5 - X) ** 2 + (yy + 0.5 - Y) ** 2) < (0.99 * R) ** 2
    assert np.all(a[inside, 0] > 0)


def pin_bruteforce_tiny():
    for seed in range(4):
        ps, cam = tiny_scene(seed)
        a = oracle.render(ps, cam)
        b = oracle.render(ps, cam, method="brute")
        assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(b).max()), seed
        assert np.abs(b).max() > 0


def pin_tiled_equals_direct():
    """Binning loses no covered pixel: the per-tile render over the member lists
    equals the direct sum, for tiles that do not divide the image."""
    rng = np.random.default_rng(11)
    n = 400
    ps = make_set(rng.uniform(0, 1, n), rng.uniform(0, 1, n), rng.uniform(0, 1, n),
                  np.exp(rng.uniform(np.log(0.002), np.log(0.08), n)), rng.uniform(0, 1, n))
    cam = front(100, 70)
    a = oracle.render(ps, cam)
    for T in (3, 8, 16, 24, 40, 64):
        b = oracle.render(ps, cam, oracle.Params(tile=T), method="tiled")
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max(), T


def pin_binning_conservative():
    """Every pixel a particle covers lies in a tile whose list holds the particle."""
    rng = np.random.default_rng(5)
    n = 150
    ps = make_set(rng.uniform(0, 1, n), rng.uniform(0, 1, n), rng.uniform(0, 1, n),
                  np.exp(rng.uniform(np.log(0.002), np.log(0.06), n)))
    cam = front(90, 60)
    for T in (5, 16, 32):
        counts, offs, mem = oracle.bins(ps, cam, oracle.Params(tile=T))
        ntx = (90 + T - 1) // T
        lists = [set(mem[offs[t]:offs[t + 1]].tolist()) for t in range(len(counts))]
        for k in range(n):
            ij = oracle.covered_pixels(ps, cam, k)
            for i, j in ij:
                assert k in lists[(j // T) * ntx + (i // T)], (T, k, i, j)


def pin_work_counts():
    """The frame's work units: covered (particle, pixel) pairs equal, for one particle
    centred on a lattice corner, the half-integer lattice points strictly inside its
    support disc, and for a random scene the pairs a per-pixel FP32 brute force finds;
    (particle, tile) pairs equal the binning's total."""
    W = H = 96
    for R_px in (0.75, 3.0, 7.25, 20.0):
        ps, cam = _single(R_px, W, H, X=48.0, Y=40.0)
        r = oracle.raster(ps, cam)
        X, Y, R = r["X"][0], r["Y"][0], r["R"][0]
        assert abs(X - 48.0) < 1e-3 and abs(Y - 40.0) < 1e-3
        k = np.arange(-64, 64) + 0.5
        lattice = int(((k[:, None] ** 2 + k[None, :] ** 2) < R * R).sum())
        w = oracle.count_work(ps, cam)
        assert w["active"] == 1 and w["pixel_pairs"] == lattice, (R_px, w, lattice)
    rng = np.random.default_rng(9)
    n = 300
    ps = make_set(rng.uniform(-0.1, 1.1, n), rng.uniform(-0.1, 1.1, n), rng.uniform(0, 1.2, n),
                  np.exp(rng.uniform(np.log(0.002), np.log(0.06), n)))
    cam = front(70, 50)
    r = oracle.raster(ps, cam)
    f = np.float32
    ii = np.arange(70, dtype=f) + f(0.5)
    jj = np.arange(50, dtype=f) + f(0.5)
    want = 0
    for q in np.nonzero(r["active"])[0]:
        X, Y, R = f(r["X"][q]), f(r["Y"][q]), f(r["R"][q])
        dx = ii[None, :] - X
        dy = jj[:, None] - Y
        want += int(((dx * dx + dy * dy) < R * R).sum())
    for T in (8, 16, 32):
        w = oracle.count_work(ps, cam, tile=T)
        assert w["active"] == int(r["active"].sum()) and w["pixel_pairs"] == want, (T, w, want)
        counts, _, _ = oracle.bins(ps, cam, oracle.Params(tile=T))
        assert w["tile_pairs"] == int(counts.sum()), (T, w)


def pin_tile_threshold():
    """Membership flips where the distance to the tile centre crosses support +
    half the tile diagonal (sqrt(2) T / 2)."""
    W = H = 128
    T = 32
    R = 0.75
    thr = R + math.sqrt(2.0) * T / 2.0
    cx, cy = 48.0, 48.0  # centre of tile (1, 1)
    xs, ys = [], []
    for eps in (-0.05, 0.05):
        d = thr + eps
        X, Y = cx - d / math.sqrt(2.0), cy - d / math.sqrt(2.0)
        w = world_for_screen(X, Y, W, H)
        xs.append(w)
    ps = make_set([w[0] for w in xs], [w[1] for w in xs], [w[2] for w in xs], [1e-6, 1e-6])
    counts, offs, mem = oracle.bins(ps, front(W, H), oracle.Params(tile=T))
    t11 = 1 * (W // T) + 1
    got = set(mem[offs[t11]:offs[t11 + 1]].tolist())
    assert got == {0}, got
    t00 = 0
    assert set(mem[offs[t00]:offs[t00 + 1]].tolist()) == {0, 1}


def pin_tile_diagram_example():
    with open(os.path.join(GOLDEN, "tile_diagram.json")) as f:
        g = json.load(f)
    W, H = g["image"]
    T = g["tile"]
    X, Y = g["screen_xy"]
    depth = g["depth"]
    x, y, z = world_for_screen(X, Y, W, H, depth)
    h = g["radius_px"] * depth / focal(H)
    ps = make_set([x], [y], [z], [h])
    counts, offs, mem = oracle.bins(ps, front(W, H), oracle.Params(tile=T))
    members = {t + 1 for t in range(len(counts)) if counts[t] > 0}
    assert members == set(g["members_paper_numbering"]), members
    # and the support itself does not reach the excluded tile
    a = oracle.render(ps, front(W, H))
    for t in g["excluded_paper_numbering"]:
        tx, ty = (t - 1) % (W // T), (t - 1) // (W // T)
        assert a[ty * T:(ty + 1) * T, tx * T:(tx + 1) * T].max() == 0.0


# ----------------------------------------------------------------------------------------
# invariants of the absorption-equals-emission sum

def _cloud(seed, n=3000):
    ps = plain_set(n, seed)
    return ps, front(80, 60)


def pin_order_invariance():
    ps, cam = _cloud(1)
    a = oracle.render(ps, cam)
    perm = np.random.default_rng(1).permutation(ps.n)
    q = make_set(ps.x[perm], ps.y[perm], ps.z[perm], ps.h[perm], ps.intensity[perm])
    b = oracle.render(q, cam)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def pin_linearity():
    ps, cam = _cloud(2)
    a = oracle.render(ps, cam)
    k = ps.n // 3
    s1 = ps.subset(np.arange(0, k))
    s2 = ps.subset(np.arange(k, ps.n))
    b = oracle.render(s1, cam) + oracle.render(s2, cam)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
    # brightness scales the deposit linearly
    c = oracle.render(ps.with_brightness([2.5]), cam)
    assert np.abs(c - 2.5 * a).max() <= 1e-12 * np.abs(c).max()


def pin_tile_size_invariance_of_image():
    ps, cam = _cloud(3)
    base = oracle.render(ps, cam, oracle.Params(tile=32), method="tiled")
    for T in (8, 16, 40, 64):
        b = oracle.render(ps, cam, oracle.Params(tile=T), method="tiled")
        assert np.abs(base - b).max() <= 1e-12 * np.abs(base).max()


def pin_rt_update_matches_closed_form():
    """Section 2.1 renders by the radiative-transfer equation along each line of sight.
    Applying the per-particle update I <- I exp(-A w) + (E/A)(1 - exp(-A w)) with A = E
    from black must give the closed form 1 - exp(-sum E w)."""
    ps, cam = _cloud(4, 1500)
    O = oracle.final(oracle.render(ps, cam))
    I = oracle.render_rt_sequential(ps, cam)
    assert np.abs(O - I).max() <= 1e-12
    assert O.max() > 0.3
    # with A = s E for a common s the same update telescopes to (1/s)(1 - exp(-s a))
    a = oracle.render(ps, cam)
    I2 = oracle.render_rt_sequential(ps, cam, absorb_scale=3.0)
    assert np.abs(I2 - (1.0 - np.exp(-3.0 * a)) / 3.0).max() <= 1e-12


def _two_species_cloud(seed, n=2400):
    """Random cloud split into two species with different colormaps."""
    rng = np.random.default_rng(seed)
    cm0 = np.array([[0.2, 0.4, 0.9], [0.9, 0.3, 0.1]], np.float32)
    cm1 = np.array([[1.0, 0.9, 0.3], [0.1, 0.8, 0.5]], np.float32)
    ps = make_set(rng.uniform(0, 1, n), rng.uniform(0, 1, n), rng.uniform(0, 1, n),
                  np.exp(rng.uniform(np.log(0.004), np.log(0.04), n)), rng.uniform(0, 1, n),
                  type_begin=[0, n // 3, n], cmaps=[cm0, cm1], betas=[0.6, 1.4])
    return ps, front(80, 60)


def pin_rt_depth_closed_forms():
    """Depth-ordered transfer with one absorption factor s for every species telescopes to
    (1/s)(1 - exp(-s a)) whatever the order (s = 1: the final transform 1 - exp(-a)), and
    to the additive sum a when nothing absorbs (s = 0)."""
    ps, cam = _two_species_cloud(3)
    a = oracle.render(ps, cam)
    assert a.max() > 0.5
    for s in (1.0, 0.4, 2.5):
        I = oracle.render_rt_depth(ps, cam, [s, s])
        assert np.abs(I - (1.0 - np.exp(-s * a)) / s).max() <= 1e-12, s
    assert np.abs(oracle.render_rt_depth(ps, cam, [1.0, 1.0]) - oracle.final(a)).max() <= 1e-12
    assert np.abs(oracle.render_rt_depth(ps, cam, [0.0, 0.0]) - a).max() <= 1e-12


def pin_rt_depth_order_two_particles():
    """Two overlapping particles of species with different absorption, both centred on one
    pixel centre (weight 1 there): the far one is applied first from black, the near one
    on top, I = I1 exp(-A2) + (E2/A2)(1 - exp(-A2)) with I1 = (E1/A1)(1 - exp(-A1)) per
    channel.  Swapping their depths swaps the roles and changes the pixel."""
    W = H = 64
    X, Y = 32.5, 30.5
    cm = np.array([[0.3, 0.6, 0.9], [0.3, 0.6, 0.9]], np.float32)
    s_abs = [2.0, 0.25]
    for far, near, depths in ((0, 1, (3.0, 1.5)), (1, 0, (1.5, 3.0))):
        pts = [world_for_screen(X, Y, W, H, depth=d) for d in depths]
        h = [(6.0 / 0.75) * d / focal(H) for d in depths]
        ps = make_set([p[0] for p in pts], [p[1] for p in pts], [p[2] for p in pts], h, [0.5, 0.5],
                      type_begin=[0, 1, 2], cmaps=[cm, cm], betas=[0.8, 1.7])
        r = oracle.raster(ps, front(W, H))
        assert r["active"].all()
        assert abs(r["X"][0] - X) < 1e-4 and abs(r["Y"][1] - Y) < 1e-4
        I = oracle.render_rt_depth(ps, front(W, H), s_abs)
        e = r["e"]
        A1, A2 = s_abs[far] * e[far], s_abs[near] * e[near]
        I1 = (e[far] / A1) * (1.0 - np.exp(-A1))
        want = I1 * np.exp(-A2) + (e[near] / A2) * (1.0 - np.exp(-A2))
        got = I[30, 32]
        assert np.abs(got - want).max() <= 1e-9 * np.abs(want).max(), (far, got, want)
    # the same two particles with their depths exchanged render a different pixel
    pair = [make_set([0.5, 0.5], [0.5, 0.5], z, [0.01, 0.01], [0.5, 0.5], type_begin=[0, 1, 2],
                     cmaps=[cm, cm], betas=[0.8, 1.7]) for z in ([0.5, 0.55], [0.55, 0.5])]
    I_a, I_b = (oracle.render_rt_depth(p, front(W, H), s_abs) for p in pair)
    assert np.abs(I_a - I_b).max() > 1e-3


def pin_rt_depth_equal_depths_in_index_order():
    """Two particles of different species at exactly the same depth on one pixel centre:
    the lower index is applied first (the reading taken for equal depths), so the pixel
    is the two-step closed form with particle 0 underneath; listing the species the other
    way round puts particle 1's species underneath."""
    W = H = 64
    X, Y = 20.5, 40.5
    cm = np.array([[0.3, 0.6, 0.9], [0.3, 0.6, 0.9]], np.float32)
    s_abs = [2.0, 0.25]
    pt = world_for_screen(X, Y, W, H, depth=2.0)
    h = (5.0 / 0.75) * 2.0 / focal(H)
    for betas in ((0.8, 1.7), (1.7, 0.8)):
        ps = make_set([pt[0]] * 2, [pt[1]] * 2, [pt[2]] * 2, [h, h], [0.5, 0.5], type_begin=[0, 1, 2],
                      cmaps=[cm, cm], betas=list(betas))
        r = oracle.raster(ps, front(W, H))
        assert r["active"].all() and r["zc"][0] == r["zc"][1]
        e = r["e"]
        A0, A1 = s_abs[0] * e[0], s_abs[1] * e[1]
        I0 = (e[0] / A0) * (1.0 - np.exp(-A0))
        want = I0 * np.exp(-A1) + (e[1] / A1) * (1.0 - np.exp(-A1))
        got = oracle.render_rt_depth(ps, front(W, H), s_abs)[40, 20]
        assert np.abs(got - want).max() <= 1e-9 * np.abs(want).max(), (betas, got, want)


def pin_rt_depth_map_closed_forms_and_slab_composition():
    """The transfer as an affine map: with unit absorption alpha = exp(-a) and beta =
    1 - exp(-a) (a the direct render's accumulation); with zero absorption alpha = 1 and
    beta = a; and the maps of two depth slabs (cameras with near / far planes at a split
    depth) compose far to near into the whole image: I = alpha_near beta_far + beta_near."""
    rng = np.random.default_rng(9)
    n = 4000
    cm = np.array([[0.2, 0.5, 0.9], [0.9, 0.4, 0.1]], np.float32)
    ps = make_set(rng.uniform(0.3, 0.7, n), rng.uniform(0.3, 0.7, n), rng.uniform(0.2, 0.8, n),
                  np.exp(rng.uniform(np.log(0.004), np.log(0.03), n)), rng.uniform(0, 1, n),
                  type_begin=[0, n // 2, n], cmaps=[cm, cm[::-1].copy()], betas=[0.05, 0.2])
    cam = front(90, 70)
    a = oracle.render(ps, cam)
    A1, B1 = oracle.render_rt_depth_map(ps, cam, [1.0, 1.0])
    assert np.abs(A1 - np.exp(-a)).max() <= 1e-12 and np.abs(B1 - (1.0 - np.exp(-a))).max() <= 1e-12
    A0, B0 = oracle.render_rt_depth_map(ps, cam, [0.0, 0.0])
    assert np.array_equal(A0, np.ones_like(A0)) and np.abs(B0 - a).max() <= 1e-12
    absorb = [2.5, 0.4]
    whole = oracle.render_rt_depth(ps, cam, absorb)
    near, far = front(90, 70), front(90, 70, z_near=2.05)
    near.z_far = 2.05
    An, Bn = oracle.render_rt_depth_map(ps, near, absorb)
    Af, Bf = oracle.render_rt_depth_map(ps, far, absorb)
    assert np.abs(Af - 1.0).max() > 0.05 and np.abs(An - 1.0).max() > 0.05  # both slabs absorb
    assert np.abs(An * Bf + Bn - whole).max() <= 1e-12
    # the same through the oracle's composition of a far-to-near list of maps
    C = oracle.compose_maps([np.concatenate([Af, Bf], -1), np.concatenate([An, Bn], -1)])
    assert np.abs(C[..., 3:] - whole).max() <= 1e-12 and np.abs(C[..., :3] - An * Af).max() <= 1e-15
    # three constant maps by hand, far to near: (a 0.5, b 1), (a 0.25, b 2), (a 2, b -1):
    # beta = 2 (0.25 * 1 + 2) - 1 = 3.5, alpha = 0.5 * 0.25 * 2 = 0.25
    consts = [(0.5, 1.0), (0.25, 2.0), (2.0, -1.0)]
    ms = [np.concatenate([np.full((2, 3, 3), a), np.full((2, 3, 3), b)], -1) for a, b in consts]
    C3 = oracle.compose_maps(ms)
    assert np.all(C3[..., :3] == 0.25) and np.all(C3[..., 3:] == 3.5)
    # the order matters: near to far gives another frame
    assert not np.allclose(oracle.compose_maps(ms[::-1])[..., 3:], 3.5)


def pin_rt_depth_lattice_is_the_full_image_restricted():
    """The lattice form leaves out only particles that cover no lattice pixel, so each of
    its pixels equals the whole image's pixel bit for bit, for several offsets and strides,
    a lattice one pixel wide, and a lattice with a ragged last row and column."""
    rng = np.random.default_rng(17)
    n = 6000
    cm = np.array([[0.2, 0.5, 0.9], [0.9, 0.4, 0.1]], np.float32)
    ps = make_set(rng.uniform(0.3, 0.7, n), rng.uniform(0.3, 0.7, n),
                  rng.choice(np.array([0.4, 0.5, 0.6], np.float32), n),
                  np.exp(rng.uniform(np.log(0.003), np.log(0.03), n)), rng.uniform(0, 1, n),
                  type_begin=[0, n // 3, n], cmaps=[cm, cm[::-1].copy()], betas=[0.05, 0.2])
    cam = front(101, 77)
    absorb = [1.7, 0.0]
    full = oracle.render_rt_depth(ps, cam, absorb)
    assert full.max() > 0.05
    for stride, ox, oy in ((1, 0, 0), (7, 3, 5), (16, 15, 0), (200, 50, 38), (10, 100, 76)):
        L = oracle.render_rt_depth_lattice(ps, cam, absorb, stride, ox, oy)
        assert np.array_equal(L, full[oy::stride, ox::stride]), (stride, ox, oy)


# ----------------------------------------------------------------------------------------
# colour (Section 2.1: scalar through a runtime colormap) and preprocessing

def _vector_set(rgb, n_scalar=0, i_log=(0, 0), i_min=None, i_max=None, beta=(0.7, 1.3)):
    """n_scalar colormap particles (species 0) then len(rgb) vector-coloured ones
    (species 1), all at the image centre."""
    n = n_scalar + len(rgb)
    ps = make_set([0.5] * n, [0.5] * n, [0.5] * n, [0.01] * n, np.linspace(0.0, 1.0, n),
                  type_begin=[0, n_scalar, n], betas=list(beta))
    ps.i_log = np.asarray(i_log, np.int32)
    ps.i_min = None if i_min is None else np.asarray(i_min, np.float32)
    ps.i_max = None if i_max is None else np.asarray(i_max, np.float32)
    full = np.zeros((n, 3), np.float32)
    full[n_scalar:] = np.asarray(rgb, np.float32)
    ps.rgb, ps.col_vector = full, np.array([0, 1], np.int32)
    return ps


def pin_vector_colour_is_the_ranged_rgb_triple():
    """Colour from a vector field: e = brightness x (C - lo) / (hi - lo) per component,
    one range over the species' three components (here r spans [0, 2], g [0, 1], b
    [0.5, 1]: a per-component range would give other values); the scalar species keeps
    its colormap colour."""
    rgb = [[0.0, 1.0, 0.5], [2.0, 0.25, 1.0], [1.0, 0.0, 0.75]]
    ps = _vector_set(rgb, n_scalar=2)
    e = oracle.raster(ps, front(16, 16))["e"]
    want = 1.3 * np.asarray(rgb, np.float64) / 2.0
    assert np.allclose(e[2:], want, rtol=0, atol=1e-7), e[2:]
    plain = ps.subset(np.arange(2))
    plain.rgb, plain.col_vector = None, None
    assert np.array_equal(e[:2], oracle.raster(plain, front(16, 16))["e"])
    # given range with clamping, and the log flag
    ps = _vector_set(rgb, i_min=[0.0, 0.5], i_max=[1.0, 1.5])
    e = oracle.raster(ps, front(16, 16))["e"]
    assert np.allclose(e, 1.3 * np.clip((np.asarray(rgb) - 0.5) / 1.0, 0, 1), rtol=0, atol=1e-7)
    rgb2 = [[1.0, np.e, np.e ** 2], [np.e ** 4, 1.0, np.e]]
    ps = _vector_set(rgb2, i_log=(0, 1))
    e = oracle.raster(ps, front(16, 16))["e"]
    assert np.allclose(e, 1.3 * np.log(np.asarray(rgb2, np.float32).astype(np.float64)) / 4.0, rtol=0,
                       atol=1e-6)


def pin_vector_colour_peak_pixel():
    """One vector-coloured particle centred on a pixel centre deposits exactly its
    emission there (weight 1), channel by channel."""
    W = H = 64
    X, Y = 20.5, 33.5
    pt = world_for_screen(X, Y, W, H, depth=2.0)
    ps = make_set([pt[0]], [pt[1]], [pt[2]], [(4.0 / 0.75) * 2.0 / focal(H)], [0.5], beta=0.9)
    ps.rgb, ps.col_vector = np.array([[0.2, 0.9, 0.5]], np.float32), np.array([1], np.int32)
    ps.i_min, ps.i_max = np.array([0.0], np.float32), np.array([1.0], np.float32)
    a = oracle.render(ps, front(W, H))
    assert np.allclose(a[33, 20], 0.9 * np.array([0.2, 0.9, 0.5]), rtol=0, atol=1e-7), a[33, 20]

def pin_colormap_special_values():
    cm = np.array([[0.0, 0.1, 0.2], [0.3, 0.5, 0.7], [1.0, 0.0, 0.5], [0.2, 0.9, 0.4],
                   [0.6, 0.6, 0.6]], np.float32)
    I = [0.0, 1.0, 0.25, 0.5, 0.75, 0.125, 0.875, 0.9999999]
    n = len(I)
    ps = make_set([0.5] * n, [0.5] * n, [0.5] * n, [0.01] * n, I, cmap=cm, beta=2.0)
    e = oracle.raster(ps, front(32, 32))["e"]
    want = [2 * cm[0], 2 * cm[4], 2 * cm[1], 2 * cm[2], 2 * cm[3], (cm[0] + cm[1]),
            (cm[3] + cm[4]), 2 * cm[4]]
    for k in range(n):
        assert np.abs(e[k] - np.asarray(want[k], np.float64)).max() < 2e-6, (k, e[k], want[k])


def pin_species_ranges():
    cma = np.array([[1.0, 0.0, 0.0], [1.0, 0.0, 0.0]], np.float32)
    cmb = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0]], np.float32)
    ps = make_set([0.5] * 4, [0.5] * 4, [0.5] * 4, [0.01] * 4, type_begin=[0, 2, 4],
                  cmaps=[cma, cmb], betas=[1.0, 3.0])
    e = oracle.raster(ps, front(16, 16))["e"]
    assert np.allclose(e[:2], [1, 0, 0]) and np.allclose(e[2:], [0, 0, 3]), e


def pin_normalisation():
    lo, hi = -3.0, 3.0
    I = np.exp(np.array([lo, hi, 0.5 * (lo + hi), lo - 1.0, hi + 1.0, lo + 1.5])).astype(np.float32)
    ps = make_set(np.zeros(6), np.zeros(6), np.zeros(6), np.ones(6), I)
    ps.i_log[:] = 1
    ps.i_min[:] = lo
    ps.i_max[:] = hi
    t = oracle.normalise(ps)
    want = [0.0, 1.0, 0.5, 0.0, 1.0, 0.25]
    assert np.abs(t - want).max() < 1e-6, t
    ps.i_min = None
    ps.i_max = None
    t = oracle.normalise(ps)
    # computed range is [lo - 1, hi + 1]
    assert t.min() == 0.0 and t.max() == 1.0 and abs(t[5] - 2.5 / 8.0) < 1e-6, t
    ps.i_log[:] = 0
    ps.intensity = np.array([2.0, 4.0, 3.0, 2.5, 4.0, 3.5], np.float32)
    t = oracle.normalise(ps)
    assert np.abs(t - [0, 1, 0.5, 0.25, 1, 0.75]).max() < 1e-12


def pin_storage_codes():
    """FP16 codes equal numpy's float16 conversion; BF16 codes equal torch's bfloat16
    conversion (both round to nearest even)."""
    rng = np.random.default_rng(3)
    v = np.concatenate([rng.uniform(-2, 2, 4000), np.exp(rng.uniform(-20, 12, 4000)),
                        [0.0, 1.0, 65504.0, 65520.0, 1e6, 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -25,
                         1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11, 5.9604645e-08, 6.1035156e-05]])
    v = v.astype(np.float32)
    q16 = oracle.quantise(v, "f16")
    with np.errstate(over="ignore"):
        ref16 = v.astype(np.float16).astype(np.float32)
    assert np.array_equal(q16, ref16), np.nonzero(q16 != ref16)
    import torch
    qb = oracle.quantise(v, "bf16")
    refb = torch.from_numpy(v).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(qb, refb), np.nonzero(qb != refb)


ALL_PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_") and callable(v)]
