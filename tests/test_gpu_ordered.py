"""Depth-ordered rendering (absorption different from emission) on the GPU: the radix
sort that orders the tile lists, and the ordered render against the FP64 oracle (needs a
GB300)."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1606_04427_gb300 import _lib, build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    assert torch.cuda.is_available()


def _sorted_on_gpu(keys, vals, lo, hi):
    k = torch.from_numpy(keys.view(np.int64)).cuda()
    v = torch.from_numpy(vals.view(np.int32)).cuda()
    _lib.check(_lib.load().splotch_debug_sort(k.data_ptr(), v.data_ptr(), keys.shape[0], lo, hi, None), "debug_sort")
    return k.cpu().numpy().view(np.uint64), v.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("n", [2, 7, 4096, 4097, 12289, 1_000_003])
def test_radix_sort_is_a_stable_sort_by_the_chosen_bits(n):
    """Sorting by key bits [lo, hi) must equal a stable sort by those bits (numpy), so
    equal keys keep their input order; many equal digits and equal keys are included."""
    rng = np.random.default_rng(n)
    tile = rng.integers(0, 300, n).astype(np.uint64)
    depth = rng.integers(0, 1 << 32, n, dtype=np.uint64)
    depth[rng.random(n) < 0.3] = 12345  # runs of equal depth keys
    keys = (tile << np.uint64(32)) | depth
    vals = np.arange(n, dtype=np.uint32)
    for lo, hi in ((0, 32), (32, 48), (0, 64), (8, 16)):
        mask = np.uint64(((1 << (hi - lo)) - 1) << lo) if hi - lo < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
        order = np.argsort(keys & mask, kind="stable")
        k, v = _sorted_on_gpu(keys.copy(), vals.copy(), lo, hi)
        assert np.array_equal(k, keys[order]), (lo, hi)
        assert np.array_equal(v, vals[order]), (lo, hi)
    # depth bits then tile bits, each pass stable: tile-major, depth-minor order
    k1, v1 = _sorted_on_gpu(keys.copy(), vals.copy(), 0, 32)
    k2, v2 = _sorted_on_gpu(k1, v1, 32, 48)
    order = np.lexsort((vals, depth, tile))
    assert np.array_equal(v2, vals[order])
