"""Particle-sharded frames across ranks (one process per GPU).

In the absorption-equals-emission mode the accumulation a is a sum over particles
(Section 2.1 additive drawing, Section 3.2.2), so a frame splits by particles: each
rank renders the accumulation of its own contiguous share of every species, the
ranks sum the images, and the final transform 1 - exp(-a) runs once on the sum.
This follows the paper's MPI model in which every task renders its particles
independently (Section 4.2.2).  The exchange is one sum-reduce of a W x H x 3 FP32
image per frame.
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
