"""The C-ABI library without a GPU: it builds for sm_103a, loads, exports every
symbol ``include/splotch.h`` declares, and its host-only logic (status strings,
defaults, FP64 camera composition, argument validation) behaves as documented.
No call here launches GPU work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
from paper_1606_04427_gb300 import _lib, build, synth
from paper_1606_04427_gb300.synth import Camera

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "splotch.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(splotch_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.SIGNATURES), set(names) ^ set(_lib.SIGNATURES)


def test_status_strings_and_defaults(lib):
    for s in range(7):
        assert lib.splotch_status_string(s)
    assert b"unknown" in lib.splotch_status_string(99)
    p = lib.splotch_default_params()
    assert (p.tile, p.rfac, p.sigma_over_R, p.r_min_px, p.block_particles, p.flags) == (0, 0.75, 0.5, 0.75, 0, 0)


def _lib_camera(lib, cam):
    m = np.zeros(12, np.float32)
    p = np.zeros(5, np.float32)
    c = _lib.camera_c(cam)
    st = lib.splotch_camera_params(C.byref(c), m.ctypes.data, p.ctypes.data)
    return st, m, p


def test_camera_composition_matches_oracle_bitwise(lib):
    """Both sides compose the camera in FP64 in the documented order and round once;
    the FP32 parameters that decide culling, coverage and binning must be identical."""
    rng = np.random.default_rng(0)
    cams = [synth.front_camera(256, 256), synth.front_camera(320, 200, 1.3, 60.0)]
    cams += synth.orbit_cameras(16, 1024, 1024)
    cams += [synth.random_camera(rng) for _ in range(200)]
    for k, cam in enumerate(cams[-50:]):  # some with a far plane
        cam.z_far = float(cam.z_near) * (2.0 + k)
    for cam in cams:
        st, m, p = _lib_camera(lib, cam)
        assert st == 0
        mo, po = oracle.camera(cam)
        assert np.array_equal(m.view(np.uint32), mo.view(np.uint32)), cam
        assert np.array_equal(p.view(np.uint32), po.view(np.uint32)), cam


@pytest.mark.parametrize("bad", [
    dict(eye=(0.5, 3.0, 0.5)),             # up parallel to the view direction
    dict(fov_deg=0.0), dict(fov_deg=180.0), dict(fov_deg=float("nan")),
    dict(eye=(0.5, 0.5, 0.5)),             # eye == lookat
    dict(z_near=0.0), dict(z_near=-1.0), dict(z_far=1e-3), dict(z_far=5e-4),
    dict(width=0), dict(height=-3),
])
def test_camera_rejections_agree(lib, bad):
    kw = dict(eye=(0.5, 0.5, 2.5), lookat=(0.5, 0.5, 0.5), up=(0.0, 1.0, 0.0), fov_deg=45.0,
              z_near=1e-3, width=8, height=8)
    kw.update(bad)
    cam = Camera(**kw)
    st, _, _ = _lib_camera(lib, cam)
    assert st == _lib.INVALID_ARG
    with pytest.raises(ValueError):
        oracle.camera(cam)


def _desc(ps, **over):
    keep = []

    def arr(a, dt):
        a = np.ascontiguousarray(a, dt)
        keep.append(a)
        return a.ctypes.data

    d = _lib.SceneDesc()
    d.n = ps.n
    d.n_types = ps.n_types
    d.type_begin = arr(ps.type_begin, np.int64)
    for k in ("x", "y", "z", "h", "intensity"):
        setattr(d, k, arr(getattr(ps, k), np.float32))
    d.storage = 0
    cms = [np.ascontiguousarray(c, np.float32) for c in ps.cmaps]
    keep += cms
    ptrs = (C.c_void_p * len(cms))(*[c.ctypes.data for c in cms])
    keep.append(ptrs)
    d.cmap_rgb = C.cast(ptrs, C.c_void_p)
    d.cmap_len = arr([c.shape[0] for c in cms], np.int32)
    d.brightness = arr(ps.brightness, np.float32)
    d.i_log = arr(ps.i_log, np.int32)
    for k, v in over.items():
        if isinstance(v, np.ndarray):
            v = arr(v, v.dtype)
        setattr(d, k, v)
    return d, keep


@pytest.mark.parametrize("over", [
    dict(n=-1), dict(n_types=0), dict(n_types=300), dict(storage=7),
    dict(type_begin=np.array([0, 5], np.int64)),         # does not end at n
    dict(type_begin=np.array([1, 64], np.int64)),        # does not start at 0
    dict(cmap_len=np.array([1], np.int32)),              # colormap with one entry
    dict(x=None), dict(brightness=None),
    dict(i_min=np.array([0.0], np.float32)),             # i_min without i_max
])
def test_create_scene_rejects_before_gpu_work(lib, over):
    ps = synth.plain_set(64, 0)
    d, keep = _desc(ps, **over)
    h = C.c_void_p()
    st = lib.splotch_create_scene(C.byref(d), C.byref(h))
    assert st == _lib.INVALID_ARG, (over, st, lib.splotch_last_error())
    assert not h.value


def test_render_rejects_null_and_bad_params(lib):
    cam = _lib.camera_c(synth.front_camera(32, 32))
    p = lib.splotch_default_params()
    assert lib.splotch_render(None, C.byref(cam), 1, C.byref(p), None, None) == _lib.INVALID_ARG
    assert lib.splotch_debug_raster(None, C.byref(cam), C.byref(p), None, None) == _lib.INVALID_ARG
    assert lib.splotch_plan_destroy(None) == 0
    assert lib.splotch_destroy(None) == 0
    assert lib.splotch_workspace_bytes(None, 10, 10, 0, 10) == -1


def test_vector_colour_without_rgb_is_rejected_before_gpu_work(lib):
    """A species flagged vector-coloured needs the per-particle RGB field."""
    ps = synth.plain_set(64, 0)
    d, keep = _desc(ps, col_vector=np.array([1], np.int32))
    h = C.c_void_p()
    assert lib.splotch_create_scene(C.byref(d), C.byref(h)) == _lib.INVALID_ARG
    assert b"rgb" in lib.splotch_last_error()
    assert not h.value


def test_entry_points_of_the_next_rows_reject_bad_arguments(lib):
    """Argument checks that run before any GPU work: the ordered render, the out-of-core
    render, the plan sequences and the sort hook."""
    cam = _lib.camera_c(synth.front_camera(32, 32))
    p = lib.splotch_default_params()
    absorb = np.array([1.0], np.float32)
    out = C.c_void_p(8)  # never dereferenced: the call fails first
    assert lib.splotch_render_ordered(None, C.byref(cam), C.byref(p), absorb.ctypes.data, out, None) == _lib.INVALID_ARG
    assert lib.splotch_plan_set_brightness(None, None, None) == _lib.INVALID_ARG
    assert lib.splotch_plan_set_colormaps(None, None, None, None) == _lib.INVALID_ARG
    keys = np.zeros(4, np.uint32)
    vals = np.zeros(4, np.uint32)
    # key width other than 4 or 8, and a bit range not a whole number of bytes
    assert lib.splotch_debug_sort(keys.ctypes.data, 3, vals.ctypes.data, 4, 0, 8, None) == _lib.INVALID_ARG
    assert lib.splotch_debug_sort(keys.ctypes.data, 4, vals.ctypes.data, 4, 0, 12, None) == _lib.INVALID_ARG
    assert lib.splotch_debug_sort(keys.ctypes.data, 4, vals.ctypes.data, 4, 0, 40, None) == _lib.INVALID_ARG
    assert lib.splotch_debug_sort(None, 8, None, -1, 0, 8, None) == _lib.INVALID_ARG


def test_far_plane_at_or_before_the_near_plane_is_rejected(lib):
    cam = synth.front_camera(32, 32)
    cam.z_far = cam.z_near
    st, _, _ = _lib_camera(lib, cam)
    assert st == _lib.INVALID_ARG
    cam.z_far = 3.0
    st, _, p = _lib_camera(lib, cam)
    assert st == 0 and p[4] == np.float32(3.0)
    cam.z_far = 0.0
    st, _, p = _lib_camera(lib, cam)
    assert st == 0 and np.isinf(p[4])


def test_two_phase_frame_and_compose_maps_reject_bad_arguments(lib):
    """The two-phase frame and the slab-map composition check their arguments before any
    GPU work: NULL scene, camera or frame, a frame rendered into NULL, and composition
    sizes and overlaps."""
    cam = _lib.camera_c(synth.front_camera(32, 32))
    p = lib.splotch_default_params()
    h = C.c_void_p()
    a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
    assert lib.splotch_frame_prepare(None, C.byref(cam), C.byref(p), None, C.byref(h), C.byref(a), C.byref(b),
                                     C.byref(c)) == _lib.INVALID_ARG
    assert not h.value
    assert lib.splotch_frame_fixed_bytes(None, C.byref(cam), C.byref(p)) == -1
    assert lib.splotch_frame_render(None, C.c_void_p(8), None) == _lib.INVALID_ARG
    assert lib.splotch_frame_destroy(None) == 0
    buf = np.zeros(6 * 10 * 2, np.float32)
    out = np.zeros(6 * 10, np.float32)
    assert lib.splotch_compose_maps(buf.ctypes.data, 0, 10, out.ctypes.data, None) == _lib.INVALID_ARG
    assert lib.splotch_compose_maps(buf.ctypes.data, 1, -1, out.ctypes.data, None) == _lib.INVALID_ARG
    assert lib.splotch_compose_maps(None, 1, 10, out.ctypes.data, None) == _lib.INVALID_ARG
    # out inside the maps it composes
    assert lib.splotch_compose_maps(buf.ctypes.data, 2, 10, buf.ctypes.data + 4 * 60, None) == _lib.INVALID_ARG
    # nothing to compose: accepted without GPU work
    assert lib.splotch_compose_maps(None, 1, 0, None, None) == 0


def test_stable_flag_value_matches_the_header(lib):
    src = open(os.path.join(ROOT, "include", "splotch.h")).read()
    m = re.search(r"SPLOTCH_STABLE\s*=\s*(\d+)", src)
    assert m and int(m.group(1)) == _lib.STABLE == 64
