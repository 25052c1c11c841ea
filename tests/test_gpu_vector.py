"""Colour from a vector field on the GPU (Section 2.1: colours come directly from a vector
input field, or from a scalar through a colormap) against the FP64 oracle (needs a GB300).

A scene with a vector-coloured species holds a per-particle emission and its tile records
carry particle indices; every splat kernel reads the emission through them.  The cases
cover the warp kernel at both square sizes and the quadrant split (tiles 8, 16, 24, 32),
the CTA kernel (tile 40), FP16 and BF16 storage, a plan with a per-view brightness sequence, the
depth-ordered render, the out-of-core render (colour ranges over the whole set) and the
argument checks."""
import numpy as np
import pytest
import torch

import oracle
from paper_1606_04427_gb300 import _lib, build, render, synth

pytestmark = pytest.mark.gpu

TOL_O = {"f32": 1e-4, "f16": 2e-3, "bf16": 2e-3}


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    assert torch.cuda.is_available()


def _vector_set(seed, n_gas=40000, n_star=15000, species=(1,)):
    ps = synth.two_species_set(n_gas, n_star, seed, grid=64).with_brightness([0.05, 0.3])
    return synth.with_vector_colour(ps, species, seed)


@pytest.mark.parametrize("tile,storage", [(8, "f32"), (16, "f32"), (16, "bf16"), (24, "f16"), (32, "f32"),
                                          (40, "f32")])
def test_vector_colour_matches_the_oracle(tile, storage):
    ps = _vector_set(10 + tile)
    cam = synth.front_camera(200, 150)
    ref = oracle.final(oracle.render(ps, cam, oracle.Params(), storage))
    sc = render.Scene(ps, storage)
    got = sc.render(cam, render.RenderParams(tile=tile)).cpu().numpy()
    err = float(np.abs(got - ref).max())
    assert err <= TOL_O[storage], (tile, storage, err)
    # the colour differs from what the colormap would give: the field is really used
    plain = synth.two_species_set(40000, 15000, 10 + tile, grid=64).with_brightness([0.05, 0.3])
    assert np.abs(ref - oracle.final(oracle.render(plain, cam, oracle.Params(), storage))).max() > 1e-2
    sc.close()


def test_every_species_vector_coloured_with_given_and_logged_ranges():
    ps = _vector_set(3, species=(0, 1))
    ps.i_log = np.array([1, 0], np.int32)
    ps.i_min = np.array([-1.0, 0.2], np.float32)
    ps.i_max = np.array([1.5, 3.0], np.float32)
    cam = synth.front_camera(160, 120)
    ref = oracle.final(oracle.render(ps, cam))
    got = render.Scene(ps, "f32").render(cam).cpu().numpy()
    assert np.abs(got - ref).max() <= TOL_O["f32"]


def test_vector_colour_in_a_plan_with_a_brightness_sequence():
    ps = _vector_set(5)
    cams = synth.orbit_cameras(4, 128, 96)
    sc = render.Scene(ps, "f16")
    plan = render.Plan(sc, cams, render.RenderParams(tile=16), graph=True)
    scale = np.array([[1.0, 1.0], [0.5, 2.0], [2.0, 0.25], [0.0, 1.0]], np.float32)
    plan.set_brightness(scale)
    out = plan.new_output()
    plan.launch(out)
    plan.check()
    for v in range(4):
        ref = oracle.final(oracle.render(ps.with_brightness(ps.brightness * scale[v]), cams[v], oracle.Params(), "f16"))
        assert np.abs(out[v].cpu().numpy() - ref).max() <= TOL_O["f16"], v
    plan.close()
    sc.close()


@pytest.mark.parametrize("absorb", [[2.0, 0.3], [8.0, 3.0]])
def test_vector_colour_in_the_depth_ordered_render(absorb):
    ps = _vector_set(7)
    cam = synth.front_camera(176, 144)
    ref = oracle.render_rt_depth(ps, cam, absorb)
    got = render.Scene(ps, "f32").render_ordered(cam, absorb, render.RenderParams(tile=16)).cpu().numpy()
    assert np.abs(got - ref).max() <= TOL_O["f32"], absorb


def test_vector_colour_out_of_core_uses_whole_set_ranges():
    ps = _vector_set(9)
    cam = synth.front_camera(160, 128)
    ref = oracle.final(oracle.render(ps, cam))
    got = render.render_streamed(ps, cam, 12000).cpu().numpy()
    assert np.abs(got - ref).max() <= TOL_O["f32"]


def test_vector_colour_argument_checks_and_memory():
    ps = _vector_set(11, 2000, 500)
    sc = render.Scene(ps, "f32")
    n, _, _, dev_bytes = sc.info()
    plain = render.Scene(synth.two_species_set(2000, 500, 11, grid=64), "f32")
    assert dev_bytes - plain.info()[3] >= 16 * n  # one FP32 emission per particle
    sc.close()
    plain.close()
    lib = _lib.load()
    bad = _vector_set(11, 2000, 500)
    bad.rgb = bad.rgb.copy()
    bad.rgb[2100, 1] = np.nan  # a star: vector-coloured
    d, keep = render._scene_desc(bad, "f32")
    h = _lib.C.c_void_p()
    assert lib.splotch_create_scene(_lib.C.byref(d), _lib.C.byref(h)) == _lib.INVALID_ARG
    bad.rgb[2100, 1] = 0.5
    bad.rgb[10, 1] = np.nan  # gas keeps its colormap: its rgb entries are not read
    d, keep = render._scene_desc(bad, "f32")
    assert lib.splotch_create_scene(_lib.C.byref(d), _lib.C.byref(h)) == _lib.OK
    lib.splotch_destroy(h)
    d, keep = render._scene_desc(bad, "f32")
    d.rgb = None
    assert lib.splotch_create_scene(_lib.C.byref(d), _lib.C.byref(h)) == _lib.INVALID_ARG
