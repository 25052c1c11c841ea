"""Multi-rank host logic on CPU (torch.distributed gloo, world size 2, spawned ranks).

The GPU render of each shard needs a GPU; here each rank's shard accumulation comes
from the CPU oracle, and the test checks what the multi-GPU path adds around the
render: every particle in exactly one shard, the image sum-reduce across ranks, the
final transform of the sum, and the benchmark's slowest-rank timing."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1606_04427_gb300 import shard, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _sharded_frame(rank, world, port, out_dir):
    _init(rank, world, port)
    import oracle
    ps = synth.two_species_set(3000, 1000, 5, grid=32).with_brightness([0.3, 0.5])
    cam = synth.front_camera(48, 40)
    mine = shard.shard_particles(ps, rank, world)
    a = torch.from_numpy(oracle.render(mine, cam))
    shard.reduce_accumulation(a)
    np.save(os.path.join(out_dir, f"a{rank}.npy"), a.numpy())
    dist.destroy_process_group()


def _slab_frame(rank, world, port, out_dir):
    """Depth slabs: rank k's slab map (here from the oracle), gathered and composed far
    to near on every rank."""
    _init(rank, world, port)
    import oracle
    ps = synth.two_species_set(3000, 1000, 6, grid=32).with_brightness([0.05, 0.3])
    cam = synth.front_camera(48, 40)
    bounds = shard.slab_bounds(cam.z_near, 1.7, 2.3, world)
    A, B = oracle.render_rt_depth_map(ps, shard.slab_camera(cam, bounds, rank), [2.0, 0.3])
    mine = torch.from_numpy(np.concatenate([A, B], -1))
    I = shard.gather_compose(mine, rank, world, compose=lambda ms: torch.from_numpy(oracle.compose_maps(ms)))
    np.save(os.path.join(out_dir, f"s{rank}.npy"), I.numpy())
    dist.destroy_process_group()


def _max_timing(rank, world, port, out_dir):
    _init(rank, world, port)
    import bench
    v = bench.max_over_ranks(10.0 + 5.0 * rank)
    np.save(os.path.join(out_dir, f"m{rank}.npy"), np.array([v]))
    dist.destroy_process_group()


def test_shard_ranges_cover_every_particle_once():
    tb = [0, 1001, 1001, 5003]
    for world in (1, 2, 3, 7):
        got = np.concatenate([shard.shard_indices(tb, r, world) for r in range(world)])
        assert np.array_equal(np.sort(got), np.arange(5003))
        for r in range(world):
            for t, (lo, hi) in enumerate(shard.shard_ranges(tb, r, world)):
                assert tb[t] <= lo <= hi <= tb[t + 1]
    with pytest.raises(ValueError):
        shard.shard_ranges(tb, 2, 2)


def test_sharded_frame_sums_to_the_whole_frame(tmp_path):
    import oracle
    world = 2
    mp.spawn(_sharded_frame, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    ps = synth.two_species_set(3000, 1000, 5, grid=32).with_brightness([0.3, 0.5])
    cam = synth.front_camera(48, 40)
    whole = oracle.render(ps, cam)
    for r in range(world):
        a = np.load(tmp_path / f"a{r}.npy")
        assert np.abs(a - whole).max() <= 1e-12 * np.abs(whole).max()
    assert np.abs(oracle.final(a) - oracle.final(whole)).max() <= 1e-12


def test_bench_step_time_is_the_slowest_rank(tmp_path):
    world = 2
    mp.spawn(_max_timing, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        assert float(np.load(tmp_path / f"m{r}.npy")[0]) == 15.0


@pytest.mark.parametrize("world", [2, 3])
def test_depth_slab_maps_compose_to_the_ordered_frame(tmp_path, world):
    """Absorption different from emission: each rank's depth slab as an affine map, all
    gathered and composed far to near, equals the whole depth-ordered frame."""
    import oracle
    mp.spawn(_slab_frame, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    ps = synth.two_species_set(3000, 1000, 6, grid=32).with_brightness([0.05, 0.3])
    whole = oracle.render_rt_depth(ps, synth.front_camera(48, 40), [2.0, 0.3])
    assert whole.max() > 0.1
    for r in range(world):
        assert np.abs(np.load(tmp_path / f"s{r}.npy") - whole).max() <= 1e-12


def test_slab_bounds_and_composition_order():
    import oracle
    b = shard.slab_bounds(1e-3, 1.5, 2.5, 4)
    assert b[0] == 1e-3 and b[-1] == 0.0 and all(x < y for x, y in zip(b[1:-1], b[2:-1]))
    with pytest.raises(ValueError):
        shard.slab_bounds(1e-3, 2.0, 1.0, 3)
    # two constant maps: far (a 0.5, b 1), near (a 0.25, b 2): I = 0.25 * 1 + 2
    far = np.concatenate([np.full((2, 2, 3), 0.5), np.full((2, 2, 3), 1.0)], -1)
    near = np.concatenate([np.full((2, 2, 3), 0.25), np.full((2, 2, 3), 2.0)], -1)
    m = oracle.compose_maps([far, near])
    assert np.allclose(m[..., :3], 0.125) and np.allclose(m[..., 3:], 2.25)
