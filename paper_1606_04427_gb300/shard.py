"""Particle-sharded frames across ranks (one process per GPU).

In the absorption-equals-emission mode the accumulation a is a sum over particles
(Section 2.1 additive drawing, Section 3.2.2), so a frame splits by particles: each
rank renders the accumulation of its own contiguous share of every species, the
ranks sum the images, and the final transform 1 - exp(-a) runs once on the sum.
This follows the paper's MPI model in which every task renders its particles
independently (Section 4.2.2).  The exchange is one sum-reduce of a W x H x 3 FP32
image per frame.

With absorption different from emission the transfer (Section 2.1) depends on the
order along each line of sight, so the frame splits by depth instead: rank k renders
the particles of depth slab k (a camera with near / far planes at consecutive bounds,
so each particle falls in exactly one slab) as the affine map I_out = alpha I_in + beta
it applies to every pixel, and the maps compose far to near.  The exchange is an
all-gather of a W x H x 6 FP32 map per rank and an ordered (non-commutative) reduction.
"""
from __future__ import annotations

import ctypes as C
from typing import List, Sequence, Tuple

import numpy as np


def shard_ranges(type_begin: Sequence[int], rank: int, world: int) -> List[Tuple[int, int]]:
    """For each species [b, e), this rank's contiguous share [b + k*len/world, ...).
    Every particle lands in exactly one rank; shares differ by at most one."""
    if not (0 <= rank < world):
        raise ValueError("rank outside [0, world)")
    out = []
    tb = [int(v) for v in type_begin]
    for t in range(len(tb) - 1):
        b, e = tb[t], tb[t + 1]
        n = e - b
        lo = b + (n * rank) // world
        hi = b + (n * (rank + 1)) // world
        out.append((lo, hi))
    return out


def shard_indices(type_begin: Sequence[int], rank: int, world: int) -> np.ndarray:
    return np.concatenate([np.arange(lo, hi, dtype=np.int64) for lo, hi in shard_ranges(type_begin, rank, world)])


def shard_particles(ps, rank: int, world: int):
    """The rank's share of a particle set (species ranges rebuilt)."""
    return ps.subset(shard_indices(ps.type_begin, rank, world))


def reduce_accumulation(a, group=None):
    """Sum the per-rank accumulation images in place (torch.distributed all-reduce)."""
    import torch.distributed as dist
    dist.all_reduce(a, op=dist.ReduceOp.SUM, group=group)
    return a


def final_transform_(a) -> None:
    """1 - exp(-a) in place on a CUDA FP32 tensor, in the library's kernel."""
    import torch
    from . import _lib
    lib = _lib.load()
    assert a.is_cuda and a.dtype == torch.float32 and a.is_contiguous()
    _lib.check(lib.splotch_final_transform(a.data_ptr(), a.numel(), torch.cuda.current_stream().cuda_stream),
               "final_transform")


def render_sharded(scene_local, cam, params=None, group=None):
    """This rank renders its shard's accumulation, the ranks sum it, and every rank
    applies the final transform to the summed image."""
    from . import render
    p = params or render.RenderParams()
    p = render.RenderParams(**{**p.__dict__, "accum": True})
    a = scene_local.render(cam, p)
    reduce_accumulation(a, group)
    final_transform_(a)
    return a


def slab_bounds(z_near: float, z_lo: float, z_hi: float, world: int) -> List[float]:
    """world + 1 ascending depth bounds: z_near, world - 1 cuts spread evenly over
    [z_lo, z_hi] (the depth extent the caller expects; it only balances the work), and 0
    (no far plane).  Slab k holds the particles with bounds[k] < z_c <= bounds[k + 1]."""
    if world < 1:
        raise ValueError("world < 1")
    cuts = [z_lo + (z_hi - z_lo) * k / world for k in range(1, world)]
    cuts = [max(c, z_near * (1.0 + 1e-6) + 1e-12 * k) for k, c in enumerate(cuts, 1)]
    for a, b in zip(cuts, cuts[1:]):
        if not b > a:
            raise ValueError("slab bounds must increase")
    return [float(z_near)] + [float(c) for c in cuts] + [0.0]


def slab_camera(cam, bounds: Sequence[float], k: int):
    """The camera of slab k: near plane bounds[k], far plane bounds[k + 1] (0: none)."""
    import dataclasses
    return dataclasses.replace(cam, z_near=float(bounds[k]), z_far=float(bounds[k + 1]))


def compose_maps(maps):
    """Compose per-slab affine maps given far to near (maps[0] the farthest slab), each an
    H x W x 6 float32 CUDA tensor (alpha rgb, beta rgb), with the library's
    splotch_compose_maps: returns the map of all of them; its beta is the frame from a
    black background."""
    import torch
    from . import _lib
    maps = list(maps)
    if not maps:
        raise ValueError("no maps")
    shape = maps[0].shape
    for m in maps:
        if not (isinstance(m, torch.Tensor) and m.is_cuda and m.dtype == torch.float32 and m.shape == shape
                and shape[-1] == 6):
            raise TypeError("compose_maps takes float32 CUDA tensors of one shape (..., 6)")
    stacked = torch.stack([m.contiguous() for m in maps])  # one buffer, farthest first
    out = torch.empty(shape, dtype=torch.float32, device=stacked.device)
    pixels = out.numel() // 6
    lib = _lib.load()
    _lib.check(lib.splotch_compose_maps(stacked.data_ptr(), len(maps), pixels, out.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream), "compose_maps")
    return out


def gather_compose(my_map, rank: int, world: int, group=None, compose=None):
    """All-gather every rank's slab map (rank k holds slab k, nearest first) and compose
    them far to near; every rank gets the frame's H x W x 3 intensity.  compose: the
    composition of a far-to-near list of maps (default: compose_maps on the GPU)."""
    import torch
    import torch.distributed as dist
    maps = [torch.empty_like(my_map) for _ in range(world)]
    dist.all_gather(maps, my_map.contiguous(), group=group)
    composed = (compose or compose_maps)(list(reversed(maps)))
    return composed[..., 3:].contiguous()


def render_ordered_sharded(scene, cam, absorb, bounds: Sequence[float], rank: int, world: int, params=None,
                           group=None):
    """Depth-sharded ordered frame: this rank renders slab `rank` of `bounds` as a map on
    its GPU, and the maps of all ranks compose far to near (see gather_compose)."""
    import dataclasses
    from .render import RenderParams
    if len(bounds) != world + 1:
        raise ValueError("need world + 1 bounds")
    pr = dataclasses.replace(params or RenderParams(), map=True)
    mine = scene.render_ordered(slab_camera(cam, bounds, rank), absorb, pr)
    return gather_compose(mine, rank, world, group)
