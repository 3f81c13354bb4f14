"""GPU grid build (histogram, scan, scatter) and dilation against the oracle:
keys, offsets, occupancy, root and ring bit-exact; CSR segments equal as
sets.  Sizes span many scan tiles and dilation tiles with ragged tails, up to
the full 226k-point scene."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_grid_equal, gpu_grid, oracle_grid_for

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k", [1, 2, 3])
def test_workload_grids(pairs, k):
    p = pairs(k)
    ctx, g = gpu_grid(p.target, L=10, voxel_size=p.voxel_size, divisions=p.grid_divisions or 16)
    og = oracle.fit_grid(p.target, p.voxel_size, p.grid_divisions)
    assert g["origin"] == og.origin and g["voxel_size"] == og.h
    assert g["inv_voxel_size"] == og.inv_h and g["dims"] == og.dims
    grid, ref = oracle_grid_for(g, p.target, 10)
    assert_grid_equal(g, ref, p.target)


@pytest.mark.parametrize("L", [0, 1, 2, 5, 15, 16, 17, 31])
def test_dilation_depths(pairs, L):
    p = pairs(1)
    ctx, g = gpu_grid(p.target, L=L, divisions=64)
    grid, ref = oracle_grid_for(g, p.target, L)
    assert_grid_equal(g, ref, p.target)


def _pts(a):
    a = np.asarray(a, np.float32)
    out = np.zeros((a.shape[0], 4), np.float32)
    out[:, :3] = a
    return out


def test_all_points_in_one_voxel():
    p = _pts(np.tile([[0.3, -0.2, 1.5]], (5000, 1)))
    ctx, g = gpu_grid(p, L=10, divisions=64)
    assert g["dims"] == (1, 1, 1)
    grid, ref = oracle_grid_for(g, p, 10)
    assert_grid_equal(g, ref, p)


def test_single_point():
    p = _pts([[1.0, 2.0, 3.0]])
    ctx, g = gpu_grid(p, L=10, divisions=64)
    grid, ref = oracle_grid_for(g, p, 10)
    assert_grid_equal(g, ref, p)


def test_points_on_voxel_faces_and_outside_an_explicit_grid():
    rng = np.random.default_rng(0)
    # multiples of h = 0.25 land exactly on voxel faces; some fall outside
    q = rng.integers(-4, 60, (4099, 3)).astype(np.float32) * 0.25
    p = _pts(q)
    ctx, g = gpu_grid(p, L=4, voxel_size=0.25, origin=(0.0, 0.0, 0.0), dims=(50, 37, 45))
    grid, ref = oracle_grid_for(g, p, 4)
    assert (ref["keys"] < 0).sum() > 100
    assert_grid_equal(g, ref, p)


def test_large_sparse_grid_more_than_2_24_voxels():
    rng = np.random.default_rng(1)
    q = rng.uniform(0, 1, (3001, 3)).astype(np.float32) * np.array([399, 299, 149], np.float32)
    p = _pts(q)
    ctx, g = gpu_grid(p, L=6, voxel_size=1.0, origin=(0.0, 0.0, 0.0), dims=(400, 300, 150))
    assert g["n_voxels"] > 2 ** 24
    grid, ref = oracle_grid_for(g, p, 6)
    assert_grid_equal(g, ref, p)


@pytest.mark.parametrize("dims", [(1, 40, 37), (45, 1, 33), (70, 29, 1), (1, 1, 300), (33, 9, 9),
                                  (36, 20, 25), (100, 12, 10), (64, 33, 5), (40, 70, 8)])
def test_thin_and_ragged_grids(dims):
    """Grids thin in one axis, ragged against the 32-voxel units, and with row
    lengths that select each store width of the dilation's fill."""
    rng = np.random.default_rng(sum(dims))
    n = 777
    q = rng.uniform(0, 1, (n, 3)) * np.array(dims) * 0.1
    p = _pts(q)
    ctx, g = gpu_grid(p, L=7, voxel_size=0.1, origin=(0.0, 0.0, 0.0), dims=dims)
    grid, ref = oracle_grid_for(g, p, 7)
    assert_grid_equal(g, ref, p)


def test_rebuild_reuses_buffers_and_stays_exact(pairs):
    """Counts return to zero after each build (the scatter decrements them),
    so repeated builds -- also of a different cloud on a smaller grid -- stay
    exact."""
    p1, p2 = pairs(2), pairs(1)
    ctx, g = gpu_grid(p1.target, L=10, divisions=128)
    import torch
    from gpu_util import to_np
    for p, div in ((p2, 128), (p1, 128), (p1, 128)):
        ctx.build_grid(torch.from_numpy(p.target).cuda())
        ctx.dilate(10)
        g = {k: to_np(v) for k, v in ctx.get_grid().items()}
        grid, ref = oracle_grid_for(g, p.target, 10)
        assert_grid_equal(g, ref, p.target)


def test_labels_follow_each_dilation_on_a_fixed_grid(pairs):
    """root/ring are rewritten only where labels were or are: a different
    cloud on the same explicit grid, and a smaller L on the same build, must
    leave no stale label behind."""
    import torch
    from gpu_util import context, to_np
    p1, p2 = pairs(1), pairs(2)
    lo = np.minimum(p1.target[:, :3].min(0), p2.target[:, :3].min(0)) - 0.05
    ctx = context(L=10, voxel_size=0.02, origin=tuple(lo), dims=(120, 110, 100))
    for p, L in ((p1, 10), (p2, 10), (p2, 3), (p1, 12), (p1, 0)):
        if L != 3:   # (p2, 3): dilate the same build again with a smaller L
            ctx.build_grid(torch.from_numpy(p.target).cuda())
        ctx.dilate(L)
        g = {k: to_np(v) for k, v in ctx.get_grid().items()}
        grid, ref = oracle_grid_for(g, p.target, L)
        assert_grid_equal(g, ref, p.target)


def test_memory_report(pairs):
    p = pairs(2)
    ctx, g = gpu_grid(p.target, L=10, divisions=128)
    rep = ctx.memory_report()
    counts = np.diff(g["offsets"].astype(np.int64))
    V = g["n_voxels"]
    assert rep["max_voxel_count"] == counts.max()
    assert rep["occupied_voxels"] == (counts > 0).sum()
    assert rep["static_bytes"] == 4 * V + 4 * (V + 1)
    assert rep["fixed_capacity_bytes"] == V * counts.max() * 4
    assert rep["paper_static_layout_bytes"] == V * 65536
    assert rep["peak_bytes"] >= rep["current_bytes"] > rep["csr_store_bytes"]
