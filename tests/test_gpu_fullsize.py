"""CUDA path against the FP64 oracle at the benchmark's full sizes, in the launch
configuration the benchmark times (default tile, FP16 or FP32 storage, CUDA-graph plan for
the batched views).  Whole frames are compared: the oracle's direct render of 100 M
particles at 2048 x 2048 takes seconds on the host cores.  Bars: max absolute per-channel
error on O <= 1e-4 (FP32 storage) and <= 2e-3 (FP16 storage, oracle fed the same rounded
attributes); the error found is printed for each result."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1606_04427_gb300 import build, render, synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

HERE = os.path.dirname(os.path.abspath(__file__))
TOL_O = {"f32": 1e-4, "f16": 2e-3}


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    assert torch.cuda.is_available()


def _brightness(key):
    with open(os.path.join(HERE, "golden", "brightness.json")) as f:
        return json.load(f)[key]


def _check(name, got, ps, cam, storage):
    ref = oracle.final(oracle.render(ps, cam, oracle.Params(), storage))
    err = float(np.abs(got - ref).max())
    print(f"\n{name}: max |O - O_oracle| = {err:.3e} (bar {TOL_O[storage]:.0e}), "
          f"mean O {float(ref.mean()):.4f}")
    assert err <= TOL_O[storage], (name, err)


def test_clustered_10M_1024_fp32_full_frame():
    ps = synth.clustered_set(10_000_000, 1).with_brightness(_brightness("clustered"))
    cam = synth.front_camera(1024, 1024)
    sc = render.Scene(ps, "f32")
    got = sc.render(cam).cpu().numpy()
    sc.close()
    _check("clustered 10M 1024^2 FP32", got, ps, cam, "f32")


def test_two_species_100M_2048_fp16_full_frame():
    ps = synth.two_species_set(70_000_000, 30_000_000, 2).with_brightness(_brightness("two_species"))
    cam = synth.front_camera(2048, 2048)
    sc = render.Scene(ps, "f16")
    got = sc.render(cam).cpu().numpy()
    sc.close()
    _check("two species 100M 2048^2 FP16", got, ps, cam, "f16")


def test_batched_64_views_20M_fp16_graph_sampled_views():
    ps = synth.clustered_set(20_000_000, 3).with_brightness(_brightness("batched"))
    cams = synth.orbit_cameras(64, 1024, 1024)
    sc = render.Scene(ps, "f16")
    plan = render.Plan(sc, cams, render.RenderParams(tile=16, block_particles=262144), graph=True)
    out = plan.new_output()
    plan.launch(out)
    plan.launch(out)  # a replay renders the same frames
    plan.check()
    for v in (0, 17, 38, 63):
        _check(f"batched view {v}", out[v].cpu().numpy(), ps, cams[v], "f16")
    plan.close()
    sc.close()


def test_clustered_20M_4096_fp16_quadrant_tiles():
    """The served stream's largest image: 4096 x 4096 needs 32-px tiles (16384 tiles),
    which the splat renders as four 16-px squares per tile; a camera at distance 1.1 from
    the box centre gives large supports and particles past the image edges."""
    ps = synth.clustered_set(20_000_000, 4).with_brightness([_brightness("served")[4] * 0.3])
    cam = synth.Camera((0.5, 0.5, 1.6), (0.5, 0.5, 0.5), (0.0, 1.0, 0.0), 45.0, 1e-3, 4096, 4096)
    sc = render.Scene(ps, "f16")
    got = sc.render(cam).cpu().numpy()
    sc.close()
    _check("clustered 20M 4096^2 FP16 (tile 32, quadrants)", got, ps, cam, "f16")


def test_two_species_100M_2048_fp16_depth_ordered_lattice():
    """The depth-ordered render (absorption 1.5 and 0.3 times the emission) of the
    benchmark frame, against the oracle's ordered transfer on a lattice of 128 x 128
    pixels (every 16th pixel from (5, 9)); the oracle applies the particles covering those
    pixels far to near, in FP64."""
    ps = synth.two_species_set(70_000_000, 30_000_000, 2).with_brightness(_brightness("two_species"))
    cam = synth.front_camera(2048, 2048)
    absorb = [1.5, 0.3]
    sc = render.Scene(ps, "f16")
    got = sc.render_ordered(cam, absorb).cpu().numpy()[9::16, 5::16]
    sc.close()
    ref = oracle.render_rt_depth_lattice(ps, cam, absorb, 16, 5, 9, storage="f16")
    err = float(np.abs(got - ref).max())
    print(f"\nordered 100M 2048^2 FP16 lattice: max |I - I_oracle| = {err:.3e} (bar 2e-03), "
          f"mean I {float(ref.mean()):.4f}")
    assert ref.mean() > 1e-2
    assert err <= TOL_O["f16"], err
