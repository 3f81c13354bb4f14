"""The voxel-histogram ablation (vicp_voxel_histogram): the warp-aggregated
design and the paper's per-block shared-memory hash (Alg. 1, key + 1 in the
packed word) both give the oracle's keys and per-voxel counts bit-exactly:
the three workloads, most points in voxel 0 (where the paper's all-zero
empty word would lose them), blocks whose 256 points all fall in distinct
voxels (full hash tables), points outside an explicit grid, and grids far
beyond the paper's 16-bit key field."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import to_np, vicp

pytestmark = pytest.mark.gpu

METHODS = [0, 1]


def _run(target, grid, method):
    v = vicp()
    t = torch.from_numpy(np.ascontiguousarray(target)).cuda()
    keys, counts = v.vicp_voxel_histogram(t, grid.origin, grid.h, grid.dims, method)
    torch.cuda.synchronize()
    return to_np(keys), to_np(counts).view(np.uint32)


def _check(target, grid, method):
    keys, counts = _run(target, grid, method)
    rk = oracle.keys(grid, target)
    V = int(np.prod(grid.dims))
    assert np.array_equal(keys, rk)
    assert np.array_equal(counts.astype(np.int64), oracle.histogram(rk, V).astype(np.int64))


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("k", [1, 2, 3])
def test_workloads(pairs, k, method):
    p = pairs(k)
    _check(p.target, oracle.fit_grid(p.target, p.voxel_size, p.grid_divisions), method)


def _pts(a):
    out = np.zeros((a.shape[0], 4), np.float32)
    out[:, :3] = a
    return out


@pytest.mark.parametrize("method", METHODS)
def test_voxel_zero_holds_most_points(method):
    rng = np.random.default_rng(2)
    q = np.concatenate([rng.uniform(0.0, 0.99, (9000, 3)), rng.uniform(0.0, 40.0, (1000, 3))])
    rng.shuffle(q)
    grid = oracle.explicit_grid((0.0, 0.0, 0.0), 1.0, (40, 40, 40))
    keys, counts = _run(_pts(q.astype(np.float32)), grid, method)
    assert counts[0] >= 9000
    _check(_pts(q.astype(np.float32)), grid, method)


@pytest.mark.parametrize("method", METHODS)
def test_full_tables_and_outside_points(method):
    """Every point in its own voxel (each block's table fills up), about a
    tenth outside the grid."""
    rng = np.random.default_rng(3)
    dims = (300, 200, 100)   # 6M voxels, far beyond 16-bit keys
    V = int(np.prod(dims))
    cells = rng.choice(V, 20000, replace=False)
    x, rem = cells % dims[0], cells // dims[0]
    y, z = rem % dims[1], rem // dims[1]
    q = np.stack([x, y, z], 1).astype(np.float64) + 0.5
    q[:2000] += np.array([400.0, 0.0, 0.0])   # outside
    rng.shuffle(q)
    _check(_pts(q.astype(np.float32)), oracle.explicit_grid((0.0, 0.0, 0.0), 1.0, dims), method)


def test_counts_are_added_to():
    v = vicp()
    rng = np.random.default_rng(4)
    t = torch.from_numpy(_pts(rng.uniform(0, 8, (5000, 3)).astype(np.float32))).cuda()
    keys, c1 = v.vicp_voxel_histogram(t, (0.0, 0.0, 0.0), 1.0, (8, 8, 8), 1)
    keys, c2 = v.vicp_voxel_histogram(t, (0.0, 0.0, 0.0), 1.0, (8, 8, 8), 0, counts=c1.clone())
    assert torch.equal(c2, 2 * c1)
