"""The allocation-free render entry point against the ordinary one (needs a GB300).

splotch_render_noalloc serves callers that may not allocate device memory while they
render (an application that owns all device memory through its own manager, a real-time
loop that allocates only at start-up).  It keeps the frame workspace in one fixed device
array inside the library, shared by every call.
These tests call it through the C ABI and compare its images with splotch_render's on
the same scene and camera, within the image bars of the parity suite, on calls made one
after the other, so that whatever one call leaves in the shared array cannot leak into
the next.  The file sorts last so that a run stopping at the first failure has already
run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest
import torch

import oracle_pins as P
from paper_1606_04427_gb300 import _lib, build, render, synth

pytestmark = pytest.mark.gpu

TOL_O = {"f32": 1e-4, "f16": 2e-3, "bf16": 2e-3}


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    assert torch.cuda.is_available()
    _lib.load()


def _nan_image(cam):
    return torch.full((cam.height, cam.width, 3), float("nan"), dtype=torch.float32, device="cuda")


def _compare(scene, cam, storage, params=None):
    want = scene.render(cam, params).cpu().numpy()
    got = scene.render_noalloc(cam, _nan_image(cam), params).cpu().numpy()
    assert np.isfinite(got).all()
    err = float(np.abs(got - want).max())
    assert err <= TOL_O[storage], f"{storage} {cam.width}x{cam.height}: max |O| error {err}"


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_two_calls_in_a_row_match_the_ordinary_render(storage):
    a = render.Scene(synth.clustered_set(60000, 1, grid=64).with_brightness([0.05]), storage)
    b = render.Scene(synth.two_species_set(40000, 15000, 2, grid=64).with_brightness([0.05, 0.3]), storage)
    # two different frames back to back, then the first again: the second call must not
    # see the first one's tile counts, and the third not the second's
    _compare(a, synth.front_camera(200, 130), storage)
    _compare(b, synth.front_camera(192, 160), storage)
    _compare(a, synth.front_camera(200, 130), storage)
    a.close()
    b.close()


def test_accumulate_flag_and_small_tiles():
    sc = render.Scene(synth.clustered_set(50000, 7, grid=64).with_brightness([0.05]), "f32")
    cam = synth.front_camera(160, 120)
    acc = render.RenderParams(accum=True, tile=16)
    want = sc.render(cam, acc).cpu().numpy()
    for _ in range(2):
        got = sc.render_noalloc(cam, _nan_image(cam), acc).cpu().numpy()
        np.testing.assert_allclose(got, want, rtol=2e-5, atol=1e-7)
    _compare(sc, synth.front_camera(97, 61), "f32", render.RenderParams(tile=8))
    sc.close()


def test_frame_beyond_the_fixed_workspace_is_rejected_and_the_next_call_is_clean():
    rng = np.random.default_rng(5)
    n = 600_000
    # every particle spans about 60 px on a 256 x 256 image: several tiles each, millions
    # of particle-tile records, more than the fixed workspace holds
    big = P.make_set(rng.uniform(0.2, 0.8, n), rng.uniform(0.2, 0.8, n), rng.uniform(0.4, 0.6, n),
                     np.full(n, 0.25), beta=1e-3)
    sc_big = render.Scene(big, "f32")
    cam = P.front(256, 256)
    with pytest.raises(_lib.SplotchError) as exc:
        sc_big.render_noalloc(cam, _nan_image(cam))
    assert exc.value.status == _lib.CAPACITY
    assert "workspace" in str(exc.value)
    sc_big.close()
    small = render.Scene(synth.clustered_set(30000, 3, grid=64).with_brightness([0.05]), "f32")
    for _ in range(2):
        _compare(small, synth.front_camera(128, 96), "f32")
    small.close()


def test_stable_lists_give_the_ordinary_render_bit_for_bit():
    """With stable tile lists the fixed-workspace render and the ordinary one build the
    same lists (ascending particle index, whatever the chunking) and cut them into the same
    work items, so their images are equal bit for bit, on two calls in a row."""
    sc = render.Scene(synth.two_species_set(30000, 12000, 6, grid=64).with_brightness([0.05, 0.3]), "f32")
    cam = synth.front_camera(150, 110)
    p = render.RenderParams(accum=True, stable=True)
    want = sc.render(cam, p)
    for _ in range(2):
        got = sc.render_noalloc(cam, _nan_image(cam), p)
        assert torch.equal(got, want)
    sc.close()


def test_bad_arguments_are_rejected_before_any_gpu_work():
    sc = render.Scene(synth.plain_set(1000, 0), "f32")
    cam = synth.front_camera(64, 64)
    out = _nan_image(cam)
    lib = _lib.load()
    c = _lib.camera_c(cam)
    assert lib.splotch_render_noalloc(None, c, None, out.data_ptr(), None) == _lib.INVALID_ARG
    assert lib.splotch_render_noalloc(sc.handle, c, None, None, None) == _lib.INVALID_ARG
    c.width = 0
    assert lib.splotch_render_noalloc(sc.handle, c, None, out.data_ptr(), None) == _lib.INVALID_ARG
    assert torch.isnan(out).all()
    sc.close()
