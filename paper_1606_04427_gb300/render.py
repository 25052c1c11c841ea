"""Python binding of the Splotch C ABI: resident scenes, frame renders, batched plans.

PyTorch supplies device memory for inputs and outputs and the CUDA stream; the
render itself (raster, tile binning, splat, final transform) runs in the CUDA
library through ``_lib``.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import check


@dataclass
class RenderParams:
    """Tile edge (0 = library default), support factor, sigma / support, minimum
    support in pixels; ``accum`` returns the accumulation a instead of 1 - exp(-a);
    ``add`` adds the accumulation to what the output holds; ``sync`` waits for the frame
    and reports device-side timeouts; ``map`` makes the depth-ordered render write the
    per-pixel affine map (alpha, beta) instead of I; ``stable`` builds every tile list in
    ascending particle index, which makes the image bitwise reproducible (the binning
    takes longer)."""
    tile: int = 0
    rfac: float = 0.75
    sigma_over_R: float = 0.5
    r_min_px: float = 0.75
    block_particles: int = 0
    accum: bool = False
    add: bool = False
    sync: bool = False
    graph: bool = False
    timing: bool = False
    map: bool = False
    stable: bool = False

    def c(self) -> _lib.RenderParamsC:
        p = _lib.RenderParamsC()
        p.tile = int(self.tile)
        p.rfac = float(self.rfac)
        p.sigma_over_R = float(self.sigma_over_R)
        p.r_min_px = float(self.r_min_px)
        p.block_particles = int(self.block_particles)
        p.flags = ((_lib.OUT_ACCUM if self.accum else 0) | (_lib.SYNC if self.sync else 0)
                   | (_lib.PLAN_GRAPH if self.graph else 0) | (_lib.TIMING if self.timing else 0)
                   | (_lib.OUT_ADD if self.add else 0) | (_lib.OUT_MAP if self.map else 0)
                   | (_lib.STABLE if self.stable else 0))
        return p


def default_tile(width: int, height: int) -> int:
    """Tile edge the library picks for tile = 0: 16 px, or the smallest edge above it in
    steps of 8 that keeps the image within 16384 tiles."""
    T = 16
    while ((width + T - 1) // T) * ((height + T - 1) // T) > 16384 and T < 64:
        T += 8
    return T


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _cams_array(cams) -> "C.Array":
    cams = list(cams)
    arr = (_lib.CameraC * len(cams))()
    for k, cam in enumerate(cams):
        arr[k] = _lib.camera_c(cam)
    return arr


def camera_params(cam):
    """The FP32 view matrix and {F, W/2, H/2, z_near, z_far} the kernels use."""
    lib = _lib.load()
    m = np.zeros(12, np.float32)
    p = np.zeros(5, np.float32)
    c = _lib.camera_c(cam)
    check(lib.splotch_camera_params(C.byref(c), m.ctypes.data, p.ctypes.data), "camera_params")
    return m, p


def last_timing():
    """Kernel durations (ms) and sizes of this thread's last render made with
    ``RenderParams(timing=True)``: {count, scan, scatter, splat, pairs, items, splits}."""
    lib = _lib.load()
    ms = np.zeros(4, np.float64)
    cnt = np.zeros(3, np.int64)
    check(lib.splotch_last_timing(ms.ctypes.data, cnt.ctypes.data), "last_timing")
    return {"count": ms[0], "scan": ms[1], "scatter": ms[2], "splat": ms[3], "pairs": int(cnt[0]),
            "items": int(cnt[1]), "splits": int(cnt[2])}


def _scene_desc(ps, storage: str, stream=None, allocator=None):
    """splotch_scene_desc of a particle set (host numpy arrays or CUDA tensors) and the
    objects that must stay alive while the library reads it."""
    keep = []

    def arr(a, dtype):
        a = np.ascontiguousarray(np.asarray(a), dtype=dtype)
        keep.append(a)
        return a.ctypes.data

    on_dev = isinstance(ps.x, torch.Tensor) and ps.x.is_cuda
    d = _lib.SceneDesc()
    n = int(ps.x.shape[0])
    d.n = n
    tb = np.asarray(ps.type_begin, np.int64)
    d.n_types = int(tb.shape[0] - 1)
    d.type_begin = arr(tb, np.int64)
    for name in ("x", "y", "z", "h", "intensity"):
        a = getattr(ps, name)
        if on_dev:
            a = a.contiguous().float()
            keep.append(a)
            setattr(d, name, a.data_ptr() if n > 0 else None)
        else:
            setattr(d, name, arr(a, np.float32) if n > 0 else None)
    d.on_device = 1 if on_dev else 0
    d.storage = _lib.STORAGE[storage]
    cms = [np.ascontiguousarray(c, np.float32) for c in ps.cmaps]
    keep.extend(cms)
    ptrs = (C.c_void_p * len(cms))(*[c.ctypes.data for c in cms])
    keep.append(ptrs)
    d.cmap_rgb = C.cast(ptrs, C.c_void_p)
    d.cmap_len = arr([c.shape[0] for c in cms], np.int32)
    d.brightness = arr(ps.brightness, np.float32)
    d.i_log = arr(ps.i_log, np.int32)
    if ps.i_min is not None and ps.i_max is not None:
        d.i_min = arr(ps.i_min, np.float32)
        d.i_max = arr(ps.i_max, np.float32)
    vec = getattr(ps, "col_vector", None)
    if vec is not None and np.any(np.asarray(vec)):
        d.col_vector = arr(vec, np.int32)
        if n > 0:
            if on_dev:
                c = torch.as_tensor(ps.rgb, device="cuda").contiguous().float().reshape(n, 3)
                keep.append(c)
                d.rgb = c.data_ptr()
            else:
                d.rgb = arr(np.asarray(ps.rgb).reshape(n, 3), np.float32)
    if allocator is not None:
        d.allocator = allocator.c()
        keep.append(allocator)
    d.stream = _stream_handle(stream)
    return d, keep


def render_streamed(ps, cam, chunk: int, params: Optional[RenderParams] = None, out: Optional[torch.Tensor] = None,
                    storage: str = "f32", stream=None, allocator=None) -> torch.Tensor:
    """Render a particle set that stays where it is (host arrays or CUDA tensors) in
    chunks of at most ``chunk`` particles, each chunk's accumulation added into one image
    (splotch_render_streamed).  Returns H x W x 3 on the device."""
    lib = _lib.load()
    d, keep = _scene_desc(ps, storage, stream, allocator)
    H, W = int(cam.height), int(cam.width)
    if out is None:
        out = torch.empty((H, W, 3), dtype=torch.float32, device="cuda")
    assert out.is_cuda and out.dtype == torch.float32 and out.is_contiguous() and out.numel() == H * W * 3
    p = (params or RenderParams()).c()
    c = _lib.camera_c(cam)
    check(lib.splotch_render_streamed(C.byref(d), int(chunk), C.byref(c), C.byref(p), out.data_ptr(),
                                      _stream_handle(stream)), "render_streamed")
    del keep
    return out


class Scene:
    """A particle set resident on the GPU (library-owned storage).

    ``ps`` has ``x, y, z, h, intensity`` (numpy float32 on the host or torch
    float32 CUDA tensors), ``type_begin``, ``cmaps``, ``brightness``, ``i_log``,
    ``i_min`` / ``i_max`` (None = computed per species)."""

    def __init__(self, ps, storage: str = "f32", stream=None, allocator=None):
        lib = _lib.load()
        self._lib = lib
        self.storage = storage
        d, keep = _scene_desc(ps, storage, stream, allocator)
        n = int(d.n)
        h = C.c_void_p()
        check(lib.splotch_create_scene(C.byref(d), C.byref(h)), "create_scene")
        self._h = h
        self._allocator = allocator
        self.n = n
        self.n_types = int(d.n_types)

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("scene destroyed")
        return self._h

    def device_bytes(self) -> int:
        b = C.c_int64()
        check(self._lib.splotch_scene_info(self.handle, None, None, None, C.byref(b)), "scene_info")
        return int(b.value)

    def render(self, cams, params: Optional[RenderParams] = None, out: Optional[torch.Tensor] = None,
               stream=None) -> torch.Tensor:
        """Render one camera (returns H x W x 3) or a list (returns V x H x W x 3)."""
        single = not isinstance(cams, (list, tuple))
        cl = [cams] if single else list(cams)
        H, W = int(cl[0].height), int(cl[0].width)
        if out is None:
            out = torch.empty((len(cl), H, W, 3), dtype=torch.float32, device="cuda")
        assert out.is_cuda and out.dtype == torch.float32 and out.is_contiguous()
        assert out.numel() == len(cl) * H * W * 3
        p = (params or RenderParams()).c()
        arr = _cams_array(cl)
        check(self._lib.splotch_render(self.handle, arr, len(cl), C.byref(p), out.data_ptr(),
                                       _stream_handle(stream)), "render")
        return out[0] if single and out.dim() == 4 else out

    def frame_fixed_bytes(self, cam, params: Optional[RenderParams] = None) -> int:
        """Device bytes the count phase of a two-phase render allocates (no GPU work)."""
        p = (params or RenderParams()).c()
        c = _lib.camera_c(cam)
        n = int(self._lib.splotch_frame_fixed_bytes(self.handle, C.byref(c), C.byref(p)))
        if n < 0:
            raise ValueError("invalid camera or parameters")
        return n

    def prepare(self, cam, params: Optional[RenderParams] = None, stream=None) -> "Frame":
        """Count phase of one view (splotch_frame_prepare): returns a :class:`Frame` that
        knows the exact device bytes its render will allocate."""
        p = (params or RenderParams()).c()
        c = _lib.camera_c(cam)
        h = C.c_void_p()
        fixed, var, pairs = C.c_int64(), C.c_int64(), C.c_int64()
        check(self._lib.splotch_frame_prepare(self.handle, C.byref(c), C.byref(p), _stream_handle(stream),
                                              C.byref(h), C.byref(fixed), C.byref(var), C.byref(pairs)),
              "frame_prepare")
        return Frame(self, h, cam, int(fixed.value), int(var.value), int(pairs.value))

    def render_noalloc(self, cam, out: torch.Tensor, params: Optional[RenderParams] = None,
                       stream=None) -> torch.Tensor:
        """Render one camera into ``out`` (H x W x 3 FP32, on the device) without any
        device allocation: the library's fixed 32 MiB workspace holds the frame.  For
        callers that may not allocate while they render.  Blocks until the frame is done.
        Calls that overlap on the GPU share that workspace and must not run at once."""
        H, W = int(cam.height), int(cam.width)
        assert out.is_cuda and out.dtype == torch.float32 and out.is_contiguous()
        assert out.numel() == H * W * 3
        p = (params or RenderParams()).c()
        c = _lib.camera_c(cam)
        check(self._lib.splotch_render_noalloc(self.handle, C.byref(c), C.byref(p), out.data_ptr(),
                                               _stream_handle(stream)), "render_noalloc")
        return out

    def render_ordered(self, cam, absorb, params: Optional[RenderParams] = None, out: Optional[torch.Tensor] = None,
                       stream=None) -> torch.Tensor:
        """Depth-ordered radiative transfer with absorption = absorb[t] x emission for
        species t, farthest particle first (splotch_render_ordered).  Returns H x W x 3, or
        with ``params.map`` H x W x 6: the affine map (alpha rgb, beta rgb) per pixel."""
        H, W = int(cam.height), int(cam.width)
        nc = 6 if (params is not None and params.map) else 3
        if out is None:
            out = torch.empty((H, W, nc), dtype=torch.float32, device="cuda")
        assert out.is_cuda and out.dtype == torch.float32 and out.is_contiguous() and out.numel() == H * W * nc
        ab = np.ascontiguousarray(np.broadcast_to(np.asarray(absorb, np.float32), (self.n_types,)))
        p = (params or RenderParams()).c()
        c = _lib.camera_c(cam)
        check(self._lib.splotch_render_ordered(self.handle, C.byref(c), C.byref(p), ab.ctypes.data, out.data_ptr(),
                                               _stream_handle(stream)), "render_ordered")
        return out

    def debug_raster(self, cam, params: Optional[RenderParams] = None, stream=None):
        out = torch.empty((8, max(1, self.n)), dtype=torch.float32, device="cuda")
        p = (params or RenderParams()).c()
        c = _lib.camera_c(cam)
        check(self._lib.splotch_debug_raster(self.handle, C.byref(c), C.byref(p), out.data_ptr(),
                                             _stream_handle(stream)), "debug_raster")
        o = out[:, : self.n]
        return {"X": o[0], "Y": o[1], "R": o[2], "zc": o[3], "e": o[4:7].T, "active": o[7] > 0.5}

    def debug_bins(self, cam, params: Optional[RenderParams] = None, capacity: Optional[int] = None,
                   stream=None):
        """(counts[n_tiles], offsets[n_tiles+1], members): the tile lists as the library
        builds them, each in ascending particle index."""
        p = (params or RenderParams()).c()
        T = p.tile if p.tile > 0 else None
        c = _lib.camera_c(cam)
        if T is None:
            T = default_tile(cam.width, cam.height)
        nt = ((cam.width + T - 1) // T) * ((cam.height + T - 1) // T)
        counts = torch.empty(nt, dtype=torch.int32, device="cuda")
        offsets = torch.empty(nt + 1, dtype=torch.int64, device="cuda")
        cap = capacity if capacity is not None else max(1024, 8 * self.n)
        members = torch.empty(cap, dtype=torch.int32, device="cuda")
        total = C.c_int64()
        st = self._lib.splotch_debug_bins(self.handle, C.byref(c), C.byref(p), counts.data_ptr(),
                                          offsets.data_ptr(), members.data_ptr(), cap, C.byref(total),
                                          _stream_handle(stream))
        if st == _lib.CAPACITY and capacity is None:
            return self.debug_bins(cam, params, capacity=int(total.value), stream=stream)
        check(st, "debug_bins")
        counts_h = counts.cpu().numpy()
        offs_h = offsets.cpu().numpy()
        mem = members[: int(total.value)].cpu().numpy()
        return counts_h, offs_h, mem

    def info(self):
        """(particle count, species count, storage code, device bytes held)."""
        n, t, st, b = C.c_int64(), C.c_int32(), C.c_int32(), C.c_int64()
        check(self._lib.splotch_scene_info(self.handle, C.byref(n), C.byref(t), C.byref(st), C.byref(b)),
              "scene_info")
        return n.value, t.value, st.value, b.value

    def workspace_bytes(self, width: int, height: int, tile: int, pairs: int) -> int:
        return int(self._lib.splotch_workspace_bytes(self.handle, int(width), int(height), int(tile),
                                                     int(pairs)))

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.splotch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Frame:
    """A prepared view (count phase done): ``fixed_bytes`` held now, ``var_bytes`` the
    exact device bytes :meth:`render` allocates, ``pairs`` its particle-tile pairs."""

    def __init__(self, scene: "Scene", handle, cam, fixed_bytes: int, var_bytes: int, pairs: int):
        self.scene = scene
        self._h = handle
        self.camera = cam
        self.fixed_bytes = fixed_bytes
        self.var_bytes = var_bytes
        self.pairs = pairs

    def render(self, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """Scatter + splat into ``out`` (H x W x 3 FP32 on the device)."""
        H, W = int(self.camera.height), int(self.camera.width)
        if out is None:
            out = torch.empty((H, W, 3), dtype=torch.float32, device="cuda")
        assert out.is_cuda and out.dtype == torch.float32 and out.is_contiguous() and out.numel() == H * W * 3
        check(self.scene._lib.splotch_frame_render(self._h, out.data_ptr(), _stream_handle(stream)), "frame_render")
        return out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self.scene._lib.splotch_frame_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """Pre-sized batched render of many views of one scene.  ``launch`` enqueues
    count, scan, scatter and one persistent splat launch over every view's work
    with no host synchronisation; with ``graph=True`` the sequence is captured into
    a CUDA graph on first launch and replayed afterwards."""

    def __init__(self, scene: Scene, cams: Sequence, params: Optional[RenderParams] = None,
                 headroom: float = 1.25, graph: bool = True, stream=None):
        self.scene = scene
        self._lib = scene._lib
        self.cams = list(cams)
        p = params or RenderParams()
        p = RenderParams(**{**p.__dict__, "graph": graph})
        self.params = p
        h = C.c_void_p()
        arr = _cams_array(self.cams)
        check(self._lib.splotch_plan_create(scene.handle, arr, len(self.cams), C.byref(p.c()),
                                            float(headroom), _stream_handle(stream), C.byref(h)),
              "plan_create")
        self._h = h
        self.V = len(self.cams)
        self.H, self.W = int(self.cams[0].height), int(self.cams[0].width)

    def info(self):
        b, t, cap = C.c_int64(), C.c_int32(), C.c_int64()
        check(self._lib.splotch_plan_info(self._h, C.byref(b), C.byref(t), C.byref(cap)), "plan_info")
        return {"device_bytes": int(b.value), "tile": int(t.value), "pair_capacity": int(cap.value)}

    def set_cameras(self, cams, stream=None):
        self.cams = list(cams)
        arr = _cams_array(self.cams)
        check(self._lib.splotch_plan_set_cameras(self._h, arr, len(self.cams), _stream_handle(stream)),
              "plan_set_cameras")

    def set_brightness(self, scale=None, stream=None) -> None:
        """Per-view emission scale per species (n_views x n_types; None resets to 1),
        applied from the next launch on, graph replays included."""
        if scale is None:
            ptr, keep = None, None
        else:
            keep = np.ascontiguousarray(np.asarray(scale, np.float32).reshape(len(self.cams), -1))
            ptr = keep.ctypes.data
        check(self._lib.splotch_plan_set_brightness(self._h, ptr, _stream_handle(stream)), "plan_set_brightness")

    def set_colormaps(self, cmaps=None, stream=None) -> None:
        """Per-view colormaps: cmaps[v][t] an (entries x 3) array for species t in view v
        (None resets every view to the scene's colormaps), from the next launch on."""
        if cmaps is None:
            check(self._lib.splotch_plan_set_colormaps(self._h, None, None, _stream_handle(stream)),
                  "plan_set_colormaps")
            return
        flat = [np.ascontiguousarray(c, np.float32).reshape(-1, 3) for row in cmaps for c in row]
        ptrs = (C.c_void_p * len(flat))(*[c.ctypes.data for c in flat])
        lens = np.array([c.shape[0] for c in flat], np.int32)
        check(self._lib.splotch_plan_set_colormaps(self._h, C.cast(ptrs, C.c_void_p), lens.ctypes.data,
                                                   _stream_handle(stream)), "plan_set_colormaps")

    def new_output(self) -> torch.Tensor:
        return torch.empty((self.V, self.H, self.W, 3), dtype=torch.float32, device="cuda")

    def launch(self, out: torch.Tensor, stream=None) -> None:
        assert out.is_cuda and out.numel() == self.V * self.H * self.W * 3 and out.is_contiguous()
        check(self._lib.splotch_plan_launch(self._h, out.data_ptr(), _stream_handle(stream)), "plan_launch")

    def check(self, stream=None) -> int:
        need = C.c_int64()
        check(self._lib.splotch_plan_check(self._h, _stream_handle(stream), C.byref(need)), "plan_check")
        return int(need.value)

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.splotch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class CallbackAllocator:
    """Device memory for scenes and workspaces from Python callables
    ``alloc(nbytes, stream) -> int`` and ``free(ptr, stream)`` (for example torch's
    caching allocator, see :func:`torch_allocator`).  A callable returning 0 makes
    the library call fail with ``SplotchError`` status OOM."""

    def __init__(self, alloc, free):
        self._alloc_py = alloc
        self._free_py = free

        def _a(ctx, nbytes, stream):
            try:
                return int(self._alloc_py(int(nbytes), stream) or 0) or None
            except Exception:
                return None

        def _f(ctx, ptr, stream):
            try:
                self._free_py(ptr, stream)
            except Exception:
                pass

        self._a = _lib.ALLOC_FN(_a)
        self._f = _lib.FREE_FN(_f)

    def c(self) -> _lib.Allocator:
        a = _lib.Allocator()
        a.alloc = self._a
        a.free = self._f
        a.ctx = None
        return a


def torch_allocator(device: int = 0) -> CallbackAllocator:
    """Workspaces from torch's caching allocator (stream-ordered per stream)."""

    def alloc(n, stream):
        return torch.cuda.caching_allocator_alloc(n, device, stream or 0)

    def free(p, stream):
        torch.cuda.caching_allocator_delete(p)

    return CallbackAllocator(alloc, free)
