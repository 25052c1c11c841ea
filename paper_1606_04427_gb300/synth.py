"""Seeded synthetic particle sets and cameras shaped like the paper's workloads.

The paper measures on a Gadget N-body SPH snapshot (50 M gas + 5 M stars for
single-node runs, 200 M + 20 M for multi-node and GPU runs), rendered as
1024^2 images along a 100-frame camera orbit and from six camera distances
from far to very close (Section 4.1, Section 4.2, Section 4.3).  That snapshot
is not available, so these generators stand in for it: a clustered N-body-like
distribution with a uniform background, SPH-style smoothing lengths that follow
the local particle spacing, lognormal intensities, a gas/star species split,
orbit cameras and random close-to-far cameras.

This module only draws inputs.  It holds none of the rendering arithmetic
(no normalisation, camera, projection, binning or splat), so the CPU oracle
and the CUDA path can both be fed from it without sharing any of the method.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

CENTRE = (0.5, 0.5, 0.5)


@dataclass
class Camera:
    """Pinhole camera: eye and look-at positions, up hint, vertical field of
    view in degrees, near-plane distance (world units), image size, and an optional
    far-plane distance (0: none)."""
    eye: Sequence[float]
    lookat: Sequence[float]
    up: Sequence[float] = (0.0, 1.0, 0.0)
    fov_deg: float = 45.0
    z_near: float = 1e-3
    width: int = 256
    height: int = 256
    z_far: float = 0.0


@dataclass
class ParticleSet:
    """Structure-of-arrays particle set.  Species are contiguous index ranges
    ``[type_begin[t], type_begin[t+1])`` (gas first, then stars)."""
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    h: np.ndarray
    intensity: np.ndarray
    type_begin: np.ndarray
    cmaps: List[np.ndarray]
    brightness: np.ndarray
    i_log: np.ndarray
    i_min: Optional[np.ndarray] = None
    i_max: Optional[np.ndarray] = None
    name: str = ""
    # colour from a vector field: per-particle RGB (n x 3, FP32) used by the species whose
    # col_vector entry is nonzero (the others keep intensity -> colormap)
    rgb: Optional[np.ndarray] = None
    col_vector: Optional[np.ndarray] = None

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_types(self) -> int:
        return int(self.type_begin.shape[0] - 1)

    def subset(self, idx: np.ndarray) -> "ParticleSet":
        """Particles ``idx`` (sorted ascending) with species ranges rebuilt."""
        idx = np.asarray(idx, dtype=np.int64)
        tb = np.searchsorted(idx, self.type_begin).astype(np.int64)
        return ParticleSet(self.x[idx], self.y[idx], self.z[idx], self.h[idx],
                           self.intensity[idx], tb, self.cmaps, self.brightness.copy(),
                           self.i_log.copy(),
                           None if self.i_min is None else self.i_min.copy(),
                           None if self.i_max is None else self.i_max.copy(),
                           self.name,
                           None if self.rgb is None else self.rgb[idx],
                           None if self.col_vector is None else self.col_vector.copy())

    def with_brightness(self, beta: Sequence[float]) -> "ParticleSet":
        out = ParticleSet(**{k: getattr(self, k) for k in self.__dataclass_fields__})
        out.brightness = np.asarray(beta, dtype=np.float32).copy()
        return out


# --------------------------------------------------------------------------------------------
# colormaps

TWO_POINT_CMAP = np.array([[0.10, 0.20, 0.60], [1.00, 0.90, 0.50]], dtype=np.float32)


def smooth_ramp_cmap(rng: np.random.Generator, n: int = 256, n_knots: int = 5) -> np.ndarray:
    """An ``n``-entry RGB ramp through ``n_knots`` random colours, joined with
    smoothstep easing so neighbouring entries differ by O(1/n)."""
    knots = rng.uniform(0.05, 1.0, size=(n_knots, 3))
    knots[0] *= 0.3  # dark low end, bright high end, like astrophysical palettes
    t = np.linspace(0.0, 1.0, n)
    seg = np.minimum((t * (n_knots - 1)).astype(np.int64), n_knots - 2)
    u = t * (n_knots - 1) - seg
    u = u * u * (3.0 - 2.0 * u)
    out = (1.0 - u)[:, None] * knots[seg] + u[:, None] * knots[seg + 1]
    return out.astype(np.float32)


# --------------------------------------------------------------------------------------------
# clustered positions and spacing-ranked smoothing lengths

@dataclass
class ClusterModel:
    centres: np.ndarray      # [K, 3]
    widths: np.ndarray       # [K]
    weights: np.ndarray      # [K], sum 1
    bg_frac: float


def draw_cluster_model(rng: np.random.Generator, n_clusters: int = 200,
                       width_range=(0.005, 0.05), zipf_a: float = 1.5,
                       bg_frac: float = 0.2) -> ClusterModel:
    centres = rng.uniform(0.0, 1.0, size=(n_clusters, 3))
    lo, hi = np.log(width_range[0]), np.log(width_range[1])
    widths = np.exp(rng.uniform(lo, hi, size=n_clusters))
    k = np.arange(1, n_clusters + 1, dtype=np.float64)
    weights = k ** (-zipf_a)
    weights /= weights.sum()
    return ClusterModel(centres, widths, weights, bg_frac)


def draw_clustered_positions(rng: np.random.Generator, n: int, model: ClusterModel,
                             width_scale: float = 1.0, chunk: int = 1 << 22) -> np.ndarray:
    """``n`` positions: a fraction ``bg_frac`` uniform in the unit box, the rest
    isotropic Gaussians around the cluster centres, wrapped periodically."""
    pos = np.empty((n, 3), dtype=np.float32)
    n_bg = int(round(model.bg_frac * n))
    is_bg = np.zeros(n, dtype=bool)
    is_bg[rng.permutation(n)[:n_bg]] = True
    cl = rng.choice(model.weights.shape[0], size=n, p=model.weights)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        c = cl[s:e]
        off = rng.standard_normal((e - s, 3)) * (model.widths[c] * width_scale)[:, None]
        p = model.centres[c] + off
        bg = is_bg[s:e]
        p[bg] = rng.uniform(0.0, 1.0, size=(int(bg.sum()), 3))
        p -= np.floor(p)
        pos[s:e] = p
    np.clip(pos, 0.0, np.float32(1.0 - 2.0 ** -24), out=pos)
    return pos


def mixture_density_grid(model: ClusterModel, width_scale: float = 1.0,
                         include_bg: bool = True, grid: int = 256) -> np.ndarray:
    """Analytic mixture density (unit mass) sampled at ``grid^3`` cell centres,
    periodic images included; separable Gaussians contract as one matrix product."""
    t = (np.arange(grid) + 0.5) / grid
    sig = model.widths * width_scale
    g = np.zeros((3, model.centres.shape[0], grid))
    for a in range(3):
        for m in (-1.0, 0.0, 1.0):
            d = t[None, :] - (model.centres[:, a][:, None] + m)
            g[a] += np.exp(-0.5 * (d / sig[:, None]) ** 2)
        g[a] /= (np.sqrt(2.0 * np.pi) * sig)[:, None]
    clf = (1.0 - model.bg_frac) if include_bg else 1.0
    A = (clf * model.weights)[:, None, None] * g[0][:, :, None] * g[1][:, None, :]
    rho = (A.reshape(A.shape[0], -1).T @ g[2]).reshape(grid, grid, grid)
    if include_bg:
        rho += model.bg_frac
    return rho.astype(np.float32)


def spacing_ranked_h(rng: np.random.Generator, pos: np.ndarray, rho_grid: np.ndarray,
                     median: float, sigma_ln: float) -> np.ndarray:
    """Draw lognormal smoothing lengths and hand them out by rank of the local
    spacing rho^(-1/3): densest particle gets the smallest h.  Keeps the stated
    marginal exactly and needs no neighbour search."""
    n = pos.shape[0]
    g = rho_grid.shape[0]
    ijk = np.minimum((pos * g).astype(np.int64), g - 1)
    rho = rho_grid[ijk[:, 0], ijk[:, 1], ijk[:, 2]]
    order = np.argsort(-rho, kind="stable")       # descending density = ascending spacing
    draws = np.sort(np.exp(rng.normal(np.log(median), sigma_ln, size=n)))
    h = np.empty(n, dtype=np.float32)
    h[order] = draws.astype(np.float32)
    return h


# --------------------------------------------------------------------------------------------
# workloads

def plain_set(n: int = 100_000, seed: int = 0) -> ParticleSet:
    """Uniform positions in the unit cube, h ~ U[0.002, 0.01], I ~ U[0, 1],
    one species, two-entry colormap."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, 1.0, size=(n, 3)).astype(np.float32)
    h = rng.uniform(0.002, 0.01, size=n).astype(np.float32)
    inten = rng.uniform(0.0, 1.0, size=n).astype(np.float32)
    return ParticleSet(np.ascontiguousarray(pos[:, 0]), np.ascontiguousarray(pos[:, 1]),
                       np.ascontiguousarray(pos[:, 2]), h, inten,
                       np.array([0, n], dtype=np.int64), [TWO_POINT_CMAP.copy()],
                       np.ones(1, np.float32), np.zeros(1, np.int32),
                       np.zeros(1, np.float32), np.ones(1, np.float32), name="plain")


def clustered_set(n: int, seed: int, h_median: float = 0.003, sigma_ln: float = 0.7,
                  grid: int = 256) -> ParticleSet:
    """One species: 200 Zipf-weighted Gaussian clusters + 20 % uniform
    background, h ranked by local spacing, lognormal intensity (log-ranged to
    [-3, 3]), two-entry colormap."""
    rng = np.random.default_rng(seed)
    model = draw_cluster_model(rng)
    pos = draw_clustered_positions(rng, n, model)
    rho = mixture_density_grid(model, grid=grid)
    h = spacing_ranked_h(rng, pos, rho, h_median, sigma_ln)
    inten = np.exp(rng.normal(0.0, 1.0, size=n)).astype(np.float32)
    return ParticleSet(np.ascontiguousarray(pos[:, 0]), np.ascontiguousarray(pos[:, 1]),
                       np.ascontiguousarray(pos[:, 2]), h, inten,
                       np.array([0, n], dtype=np.int64), [TWO_POINT_CMAP.copy()],
                       np.ones(1, np.float32), np.ones(1, np.int32),
                       np.full(1, -3.0, np.float32), np.full(1, 3.0, np.float32),
                       name="clustered")


def two_species_set(n_gas: int, n_star: int, seed: int, grid: int = 256) -> ParticleSet:
    """Gas drawn as :func:`clustered_set`; stars from the same centres with
    widths x 0.2, no background and h five times smaller; one 256-entry ramp
    colormap per species."""
    rng = np.random.default_rng(seed)
    model = draw_cluster_model(rng)
    gas = draw_clustered_positions(rng, n_gas, model)
    h_gas = spacing_ranked_h(rng, gas, mixture_density_grid(model, grid=grid), 0.003, 0.7)
    star_model = ClusterModel(model.centres, model.widths, model.weights, 0.0)
    stars = draw_clustered_positions(rng, n_star, star_model, width_scale=0.2)
    h_star = spacing_ranked_h(rng, stars,
                              mixture_density_grid(star_model, 0.2, include_bg=False, grid=grid),
                              0.0006, 0.7)
    inten = np.exp(rng.normal(0.0, 1.0, size=n_gas + n_star)).astype(np.float32)
    cmaps = [smooth_ramp_cmap(rng), smooth_ramp_cmap(rng)]
    pos = np.concatenate([gas, stars])
    del gas, stars
    return ParticleSet(np.ascontiguousarray(pos[:, 0]), np.ascontiguousarray(pos[:, 1]),
                       np.ascontiguousarray(pos[:, 2]), np.concatenate([h_gas, h_star]), inten,
                       np.array([0, n_gas, n_gas + n_star], dtype=np.int64), cmaps,
                       np.ones(2, np.float32), np.ones(2, np.int32),
                       np.full(2, -3.0, np.float32), np.full(2, 3.0, np.float32),
                       name="two_species")


def with_vector_colour(ps: ParticleSet, species: Sequence[int], seed: int = 0) -> ParticleSet:
    """The same set with the given species coloured from a vector field (Section 2.1):
    a per-particle RGB triple, here a smooth positive field of position with lognormal
    scatter (like velocity or chemical-abundance components mapped to colour), drawn for
    every particle; the other species keep their colormap."""
    rng = np.random.default_rng(seed)
    n = ps.n
    k = rng.uniform(2.0, 6.0, size=(3, 3))
    ph = rng.uniform(0.0, 2.0 * np.pi, size=3)
    pos = np.stack([ps.x, ps.y, ps.z], axis=1).astype(np.float32)
    rgb = np.empty((n, 3), np.float32)
    for c in range(3):
        rgb[:, c] = 1.2 + np.sin(pos @ k[c].astype(np.float32) * np.float32(2.0 * np.pi) + np.float32(ph[c]))
    rgb *= np.exp(rng.normal(0.0, 0.25, size=(n, 3))).astype(np.float32)
    out = ParticleSet(**{f: getattr(ps, f) for f in ps.__dataclass_fields__})
    out.rgb = rgb
    vec = np.zeros(ps.n_types, np.int32)
    vec[list(species)] = 1
    out.col_vector = vec
    return out


def front_camera(width: int, height: int, distance: float = 2.0, fov_deg: float = 45.0) -> Camera:
    """Camera on the +z axis at ``distance`` from the box centre, looking at it."""
    c = CENTRE
    return Camera((c[0], c[1], c[2] + distance), c, (0.0, 1.0, 0.0), fov_deg, 1e-3, width, height)


def orbit_cameras(n_views: int, width: int, height: int, radius: float = 2.0) -> List[Camera]:
    """``n_views`` cameras on a horizontal circle of ``radius`` around the box
    centre, angle 2 pi k / n_views, all looking at the centre."""
    c = CENTRE
    out = []
    for k in range(n_views):
        th = 2.0 * math.pi * k / n_views
        eye = (c[0] + radius * math.sin(th), c[1], c[2] + radius * math.cos(th))
        out.append(Camera(eye, c, (0.0, 1.0, 0.0), 45.0, 1e-3, width, height))
    return out


def random_camera(rng: np.random.Generator, sizes=(512, 1024, 2048, 4096),
                  dist_range=(0.6, 4.0)) -> Camera:
    """Direction uniform on the sphere, distance log-uniform, square image of a
    size drawn from ``sizes``; cameras inside the box are included."""
    v = rng.standard_normal(3)
    v /= np.linalg.norm(v)
    d = math.exp(rng.uniform(math.log(dist_range[0]), math.log(dist_range[1])))
    c = np.asarray(CENTRE)
    eye = c + d * v
    up = (0.0, 1.0, 0.0) if abs(v[1]) < 0.95 else (1.0, 0.0, 0.0)
    s = int(rng.choice(np.asarray(sizes)))
    return Camera(tuple(float(a) for a in eye), CENTRE, up, 45.0, 1e-3, s, s)


def served_set_sizes(n_sets: int = 8, n_min: float = 1e6, n_max: float = 2e8) -> List[int]:
    """Geometric sizes n_min * (n_max/n_min)^(k/(n_sets-1))."""
    return [int(round(n_min * (n_max / n_min) ** (k / (n_sets - 1)))) for k in range(n_sets)]


@dataclass
class Request:
    set_index: int
    camera: Camera
    arrival_s: float


def poisson_requests(rng: np.random.Generator, n_requests: int, rate_per_s: float,
                     n_sets: int, sizes=(512, 1024, 2048, 4096)) -> List[Request]:
    """Render requests with exponential inter-arrival times, a uniformly chosen
    resident set and a random camera each."""
    t = 0.0
    out = []
    for _ in range(n_requests):
        t += rng.exponential(1.0 / rate_per_s)
        out.append(Request(int(rng.integers(0, n_sets)), random_camera(rng, sizes), t))
    return out
