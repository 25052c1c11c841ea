"""Python marshalling for the FP64 CPU oracle (``splotch_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  All arithmetic lives in
the C file; this module converts numpy arrays to pointers and back.  It imports
nothing from the CUDA package.

Functions take a *particle set* object with attributes ``x, y, z, h,
intensity`` (float32 arrays), ``type_begin`` (int64), ``cmaps`` (list of
``[n_t, 3]`` float32), ``brightness``, ``i_log``, ``i_min``, ``i_max``
(per species; ``i_min``/``i_max`` may be None = computed), and a *camera*
object with ``eye, lookat, up, fov_deg, z_near, width, height``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "splotch_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

STORAGE = {"f32": 0, "f16": 1, "bf16": 2}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, IEEE FP32/FP64, no contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(path: str):
    """Load an oracle shared library and declare its C signatures."""
    lib = C.CDLL(path)
    P = C.c_void_p
    i64, i32, f32, f64 = C.c_int64, C.c_int, C.c_float, C.c_double
    scene = [i64, P, P, P, P, P, i32, P, P, P, P, P, P, i32, i32, f32, f32, f64, P, P]
    lib.orc_camera.argtypes = [P, P, P, f64, f64, f64, i32, i32, P, P]
    lib.orc_camera.restype = i32
    lib.orc_normalise.argtypes = [i64, P, i32, i32, f64, f64, i32, P]
    lib.orc_quantise_f32.argtypes = [i64, P, P, i32]
    lib.orc_to_f16.argtypes = [f64]
    lib.orc_to_f16.restype = f64
    lib.orc_to_bf16.argtypes = [f64]
    lib.orc_to_bf16.restype = f64
    lib.orc_raster.argtypes = scene + [P, P, P]
    lib.orc_render.argtypes = scene + [P]
    lib.orc_render_bruteforce.argtypes = scene + [P]
    lib.orc_render_rt_sequential.argtypes = scene + [f64, P]
    lib.orc_render_tiled.argtypes = scene + [i32, P]
    lib.orc_bin.argtypes = scene + [i32, P, P, P, i64, P]
    lib.orc_covered_pixels.argtypes = scene + [i64, P, i64]
    lib.orc_covered_pixels.restype = i64
    lib.orc_render_rt_depth.argtypes = scene + [P, P]
    lib.orc_render_rt_depth.restype = i32
    lib.orc_render_rt_depth_lattice.argtypes = scene + [P, i32, i32, i32, P]
    lib.orc_render_rt_depth_map.argtypes = scene + [P, P, P]
    lib.orc_render_rt_depth_map.restype = i32
    lib.orc_render_rt_depth_lattice.restype = i32
    lib.orc_count_work.argtypes = scene + [i32, P]
    lib.orc_count_work.restype = i32
    lib.orc_final.argtypes = [i64, P, P]
    lib.orc_num_threads.restype = i32
    lib.orc_set_threads.argtypes = [i32]
    for f in ("orc_raster", "orc_render", "orc_render_bruteforce", "orc_render_rt_sequential",
              "orc_render_tiled", "orc_bin"):
        getattr(lib, f).restype = i32
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
        return _lib


_active = threading.local()


def _cur():
    """The library the module functions call: the built oracle, or a variant made
    current by :func:`using` (the mutation tests plant mistakes that way)."""
    lib = getattr(_active, "lib", None)
    return lib if lib is not None else _load()


class using:
    """Context manager: route this thread's oracle calls to another build of
    ``splotch_oracle.c`` (e.g. one compiled from a deliberately altered copy)."""

    def __init__(self, lib):
        self.lib = lib

    def __enter__(self):
        self.prev = getattr(_active, "lib", None)
        _active.lib = self.lib
        return self.lib

    def __exit__(self, *exc):
        _active.lib = self.prev


def build_variant(source_text: str, out_path: str):
    """Compile C source text (a variant of the oracle) to ``out_path`` and load it."""
    src_path = out_path + ".c"
    with open(src_path, "w") as f:
        f.write(source_text)
    cmd = ["gcc", "-O1", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-w", "-o", out_path, src_path, "-lm"]
    subprocess.run(cmd, check=True)
    return _bind(out_path)


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def _ptr(a: np.ndarray):
    return C.c_void_p(a.ctypes.data)


def num_threads() -> int:
    return int(_cur().orc_num_threads())


def set_threads(n: int) -> None:
    _cur().orc_set_threads(int(n))


@dataclass
class Params:
    tile: int = 32
    rfac: float = 0.75
    sigma_over_R: float = 0.5
    r_min_px: float = 0.75


def camera(cam):
    """FP32 3x4 view matrix and {F, cx, cy, z_near, z_far}; raises ValueError when rejected.
    A camera without z_far (or with z_far 0 / infinite) has no far plane."""
    lib = _cur()
    m = np.zeros(12, np.float32)
    p = np.zeros(5, np.float32)
    e = np.asarray(cam.eye, np.float64)
    l = np.asarray(cam.lookat, np.float64)
    u = np.asarray(cam.up, np.float64)
    rc = lib.orc_camera(_ptr(e), _ptr(l), _ptr(u), float(cam.fov_deg), float(cam.z_near),
                        float(getattr(cam, "z_far", 0.0) or 0.0), int(cam.width), int(cam.height), _ptr(m), _ptr(p))
    if rc != 0:
        raise ValueError("camera rejected")
    return m, p


def to_f16(v: float) -> float:
    return float(_cur().orc_to_f16(float(v)))


def to_bf16(v: float) -> float:
    return float(_cur().orc_to_bf16(float(v)))


def quantise(a: np.ndarray, storage: str) -> np.ndarray:
    a = np.ascontiguousarray(a, np.float32)
    out = np.empty_like(a)
    _cur().orc_quantise_f32(a.shape[0], _ptr(a), _ptr(out), STORAGE[storage])
    return out


def normalise(ps, storage: str = "f32") -> np.ndarray:
    """Normalised intensity per particle, FP64 (after storage rounding)."""
    lib = _cur()
    out = np.empty(ps.n if hasattr(ps, "n") else ps.x.shape[0], np.float64)
    tb = np.asarray(ps.type_begin, np.int64)
    for t in range(tb.shape[0] - 1):
        s, e = int(tb[t]), int(tb[t + 1])
        I = np.ascontiguousarray(ps.intensity[s:e], np.float32)
        seg = np.empty(e - s, np.float64)
        given = ps.i_min is not None and ps.i_max is not None
        lo = float(ps.i_min[t]) if given else 0.0
        hi = float(ps.i_max[t]) if given else 0.0
        lib.orc_normalise(e - s, _ptr(I), int(ps.i_log[t]), int(given), lo, hi,
                          STORAGE[storage], _ptr(seg))
        out[s:e] = seg
    return out


def normalise_rgb(ps):
    """Normalised colour components (n x 3, FP64) of the vector-coloured species, zeros
    elsewhere; None when the set has no vector-coloured species.  A species' three
    components share one range (given, or their joint min / max) and its log flag."""
    vec = getattr(ps, "col_vector", None)
    if vec is None or not np.any(np.asarray(vec)):
        return None
    lib = _cur()
    n = int(ps.x.shape[0])
    out = np.zeros((n, 3), np.float64)
    tb = np.asarray(ps.type_begin, np.int64)
    for t in range(tb.shape[0] - 1):
        if not vec[t]:
            continue
        s, e = int(tb[t]), int(tb[t + 1])
        comp = np.ascontiguousarray(ps.rgb[s:e], np.float32).reshape(-1)
        seg = np.empty(comp.shape[0], np.float64)
        given = ps.i_min is not None and ps.i_max is not None
        lo = float(ps.i_min[t]) if given else 0.0
        hi = float(ps.i_max[t]) if given else 0.0
        lib.orc_normalise(comp.shape[0], _ptr(comp), int(ps.i_log[t]), int(given), lo, hi, 0, _ptr(seg))
        out[s:e] = seg.reshape(-1, 3)
    return out


class _Scene:
    """Keeps the marshalled arrays alive for one oracle call."""

    def __init__(self, ps, cam, params: Params, storage: str):
        self.n = int(ps.x.shape[0])
        q = (lambda a: quantise(a, storage)) if storage != "f32" else (
            lambda a: np.ascontiguousarray(a, np.float32))
        self.x, self.y, self.z, self.h = q(ps.x), q(ps.y), q(ps.z), q(ps.h)
        self.It = normalise(ps, storage)
        self.tb = np.ascontiguousarray(ps.type_begin, np.int64)
        self.nt = int(self.tb.shape[0] - 1)
        self.cm = [np.ascontiguousarray(c, np.float32) for c in ps.cmaps]
        self.cm_ptrs = (C.c_void_p * self.nt)(*[c.ctypes.data for c in self.cm])
        self.cm_len = np.array([c.shape[0] for c in self.cm], np.int32)
        self.beta = np.ascontiguousarray(ps.brightness, np.float64)
        self.m, self.p = camera(cam)
        self.W, self.H = int(cam.width), int(cam.height)
        self.params = params
        self.rgb = normalise_rgb(ps)
        self.vec = (np.ascontiguousarray(ps.col_vector, np.int32) if self.rgb is not None else None)

    def args(self):
        pr = self.params
        return [self.n, _ptr(self.x), _ptr(self.y), _ptr(self.z), _ptr(self.h), _ptr(self.It),
                self.nt, _ptr(self.tb), C.cast(self.cm_ptrs, C.c_void_p), _ptr(self.cm_len),
                _ptr(self.beta), _ptr(self.m), _ptr(self.p), self.W, self.H,
                float(pr.rfac), float(pr.r_min_px), float(pr.sigma_over_R),
                None if self.rgb is None else _ptr(self.rgb), None if self.vec is None else _ptr(self.vec)]


def raster(ps, cam, params: Params = Params(), storage: str = "f32"):
    """Dict with X, Y, R, zc (FP32 values as FP64), e [n, 3] (FP64), active (bool), box [n, 4]."""
    s = _Scene(ps, cam, params, storage)
    out = np.zeros((7, s.n), np.float64)
    act = np.zeros(s.n, np.int32)
    box = np.zeros((s.n, 4), np.int32)
    rc = _cur().orc_raster(*s.args(), _ptr(out), _ptr(act), _ptr(box))
    assert rc == 0
    return {"X": out[0], "Y": out[1], "R": out[2], "zc": out[3], "e": out[4:7].T.copy(),
            "active": act.astype(bool), "box": box}


def render(ps, cam, params: Params = Params(), storage: str = "f32", method: str = "direct"):
    """Pre-transform accumulation a (H x W x 3, FP64).  method: direct | tiled | brute."""
    s = _Scene(ps, cam, params, storage)
    a = np.zeros((s.H, s.W, 3), np.float64)
    lib = _cur()
    if method == "direct":
        rc = lib.orc_render(*s.args(), _ptr(a))
    elif method == "tiled":
        rc = lib.orc_render_tiled(*s.args(), int(params.tile), _ptr(a))
    elif method == "brute":
        rc = lib.orc_render_bruteforce(*s.args(), _ptr(a))
    else:
        raise ValueError(method)
    assert rc == 0, rc
    return a


def render_rt_depth(ps, cam, absorb, params: Params = Params(), storage: str = "f32"):
    """Image from the radiative-transfer update applied in depth order, farthest first,
    with absorption = absorb[t] x emission for species t (H x W x 3, FP64)."""
    s = _Scene(ps, cam, params, storage)
    ab = np.ascontiguousarray(np.broadcast_to(np.asarray(absorb, np.float64), (s.nt,)))
    I = np.zeros((s.H, s.W, 3), np.float64)
    rc = _cur().orc_render_rt_depth(*s.args(), _ptr(ab), _ptr(I))
    assert rc == 0
    return I


def render_rt_depth_map(ps, cam, absorb, params: Params = Params(), storage: str = "f32"):
    """(alpha, beta), each H x W x 3 FP64: the depth-ordered transfer as the affine map
    I_out = alpha I_in + beta it applies to each pixel (beta = render_rt_depth)."""
    s = _Scene(ps, cam, params, storage)
    ab = np.ascontiguousarray(np.broadcast_to(np.asarray(absorb, np.float64), (s.nt,)))
    A = np.ones((s.H, s.W, 3), np.float64)
    B = np.zeros((s.H, s.W, 3), np.float64)
    rc = _cur().orc_render_rt_depth_map(*s.args(), _ptr(ab), _ptr(A), _ptr(B))
    assert rc == 0
    return A, B


def compose_maps(maps):
    """Composition of per-pixel affine maps I_out = alpha I_in + beta given far to near
    (maps[0] the farthest), each H x W x 6 (alpha rgb, beta rgb), FP64: the transfer of
    Section 2.1 takes the farther material first, so a nearer map applies after a farther
    one, beta <- alpha_near beta + beta_near and alpha <- alpha_near alpha."""
    maps = [np.asarray(m, np.float64) for m in maps]
    if not maps:
        raise ValueError("no maps")
    alpha = maps[0][..., :3].copy()
    beta = maps[0][..., 3:].copy()
    for m in maps[1:]:
        beta = m[..., :3] * beta + m[..., 3:]
        alpha = m[..., :3] * alpha
    return np.concatenate([alpha, beta], -1)


def render_rt_depth_lattice(ps, cam, absorb, stride: int, ox: int = 0, oy: int = 0, params: Params = Params(),
                            storage: str = "f32"):
    """render_rt_depth at the pixels (ox + stride a, oy + stride b) only: equal to
    render_rt_depth(...)[oy::stride, ox::stride], for images too large to render whole."""
    s = _Scene(ps, cam, params, storage)
    ab = np.ascontiguousarray(np.broadcast_to(np.asarray(absorb, np.float64), (s.nt,)))
    nx, ny = -(-(s.W - ox) // stride), -(-(s.H - oy) // stride)
    L = np.zeros((ny, nx, 3), np.float64)
    rc = _cur().orc_render_rt_depth_lattice(*s.args(), _ptr(ab), ox, oy, stride, _ptr(L))
    assert rc == 0
    return L


def render_rt_sequential(ps, cam, params: Params = Params(), storage: str = "f32",
                         absorb_scale: float = 1.0):
    """Image from the per-particle radiative-transfer update (H x W x 3, FP64)."""
    s = _Scene(ps, cam, params, storage)
    I = np.zeros((s.H, s.W, 3), np.float64)
    rc = _cur().orc_render_rt_sequential(*s.args(), float(absorb_scale), _ptr(I))
    assert rc == 0
    return I


def final(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, np.float64)
    O = np.empty_like(a)
    _cur().orc_final(a.size, _ptr(a), _ptr(O))
    return O


def image(ps, cam, params: Params = Params(), storage: str = "f32"):
    """(a, O): accumulation and final image."""
    a = render(ps, cam, params, storage)
    return a, final(a)


def bins(ps, cam, params: Params = Params(), storage: str = "f32"):
    """(counts[n_tiles] int32, offsets[n_tiles+1] int64, members int32 ascending per tile)."""
    s = _Scene(ps, cam, params, storage)
    T = int(params.tile)
    nt = ((s.W + T - 1) // T) * ((s.H + T - 1) // T)
    counts = np.zeros(nt, np.int32)
    offs = np.zeros(nt + 1, np.int64)
    total = np.zeros(1, np.int64)
    lib = _cur()
    rc = lib.orc_bin(*s.args(), T, _ptr(counts), _ptr(offs), None, 0, _ptr(total))
    assert rc == 0
    mem = np.zeros(max(1, int(total[0])), np.int32)
    rc = lib.orc_bin(*s.args(), T, _ptr(counts), _ptr(offs), _ptr(mem), mem.shape[0], _ptr(total))
    assert rc == 0
    return counts, offs, mem[: int(total[0])]


def count_work(ps, cam, params: Params = Params(), storage: str = "f32", tile: int = 0) -> dict:
    """Active particles, covered (particle, pixel) pairs and, for tile > 0, (particle,
    tile) pairs of one frame."""
    s = _Scene(ps, cam, params, storage)
    out = np.zeros(3, np.int64)
    rc = _cur().orc_count_work(*s.args(), int(tile), _ptr(out))
    assert rc == 0, rc
    return {"active": int(out[0]), "pixel_pairs": int(out[1]), "tile_pairs": int(out[2])}


def covered_pixels(ps, cam, k: int, params: Params = Params(), storage: str = "f32") -> np.ndarray:
    """[(i, j)] pixels covered by particle k."""
    s = _Scene(ps, cam, params, storage)
    lib = _cur()
    cnt = lib.orc_covered_pixels(*s.args(), int(k), None, 0)
    ij = np.zeros((max(1, cnt), 2), np.int32)
    lib.orc_covered_pixels(*s.args(), int(k), _ptr(ij), cnt)
    return ij[:cnt]
