"""The fixed-capacity voxel store (vicp_fixed_build / vicp_fixed_correspond)
against the CSR store: with a capacity of the largest voxel count nothing is
dropped and every neighbour, distance and global-search count equals
vicp_correspond's bit for bit (all three workloads, the scene included); with
a smaller capacity the dropped points equal sum(max(0, count - C)) over the
oracle's histogram, queries whose root voxel kept all its points are
unchanged, and the others get a stored point no closer than the CSR answer."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import gpu_grid, to_np, vicp
from paper_2512_04996_gb300.synth import random_rigid

pytestmark = pytest.mark.gpu


def _searches(ctx, src, T):
    s = torch.from_numpy(np.ascontiguousarray(src)).cuda()
    pose = torch.from_numpy(np.ascontiguousarray(T, dtype=np.float64)).cuda()
    a = [to_np(x) for x in ctx.correspond(s, pose)]
    b = [to_np(x) for x in ctx.fixed_correspond(s, pose)]
    return a, b


@pytest.mark.parametrize("k", [1, 2, 3])
def test_capacity_of_the_largest_voxel_equals_csr(pairs, k):
    p = pairs(k)
    ctx, g = gpu_grid(p.target, L=10, voxel_size=p.voxel_size, divisions=p.grid_divisions)
    rep = ctx.memory_report()
    C = rep["max_voxel_count"]
    over, nbytes = ctx.fixed_build(g["_target"], C)
    assert over == 0
    assert nbytes == g["n_voxels"] * C * 16 + 4 * g["n_voxels"]
    for T in (np.eye(4), p.T_gt, random_rigid(np.random.default_rng(k), 20.0, 0.2)):
        (nn, d2, nf), (fnn, fd2, fnf) = _searches(ctx, p.source, T)
        assert np.array_equal(nn, fnn) and np.array_equal(d2.view(np.uint32), fd2.view(np.uint32))
        assert int(nf[0]) == int(fnf[0])


def test_small_capacity_drops_and_approximates(pairs):
    p = pairs(2)
    ctx, g = gpu_grid(p.target, L=10, voxel_size=p.voxel_size, divisions=p.grid_divisions)
    counts = np.diff(g["offsets"].astype(np.int64))
    C = max(1, int(counts.max()) // 4)
    over, _ = ctx.fixed_build(g["_target"], C)
    assert over == int(np.maximum(counts - C, 0).sum()) and over > 0
    (nn, d2, nf), (fnn, fd2, fnf) = _searches(ctx, p.source, p.T_gt)
    # the root voxel of each query, from the CSR grid
    from gpu_util import transform_f32
    grid = oracle.Grid(g["origin"], g["voxel_size"], g["inv_voxel_size"], g["dims"])
    keys = oracle.keys(grid, transform_f32(p.T_gt, p.source))
    root = np.where(keys >= 0, g["root"][np.maximum(keys, 0)], -1)
    full = (root >= 0) & (counts[np.maximum(root, 0)] <= C)
    assert full.sum() > 0 and (~full & (root >= 0)).sum() > 0
    assert np.array_equal(nn[full], fnn[full]) and np.array_equal(d2[full], fd2[full])
    part = (root >= 0) & ~full
    assert np.all((fnn[part] >= 0) & (fnn[part] < p.target.shape[0]))
    assert np.all(fd2[part] >= d2[part])
    # the global searches are the same queries
    assert np.array_equal(nn[root < 0], fnn[root < 0])


def test_fixed_store_argument_checks(pairs):
    v = vicp()
    p = pairs(1)
    ctx = v.Context(v.default_params(grid_divisions=64))
    t = torch.from_numpy(p.target).cuda()
    with pytest.raises(v.VicpError) as e:
        ctx.fixed_build(t, 8)
    assert e.value.status == v.VICP_ERR_STATE
    ctx.build_grid(t)
    with pytest.raises(v.VicpError) as e:
        ctx.fixed_build(t, 0)
    assert e.value.status == v.VICP_ERR_INVALID
    with pytest.raises(v.VicpError) as e:
        ctx.fixed_build(t, 1 << 20)   # V * C >= 2^32
    assert e.value.status == v.VICP_ERR_GRID_TOO_LARGE
    ctx.fixed_build(t, 64)
    with pytest.raises(v.VicpError) as e:   # no dilation yet
        ctx.fixed_correspond(torch.from_numpy(p.source).cuda(), torch.eye(4, dtype=torch.float64, device="cuda"))
    assert e.value.status == v.VICP_ERR_STATE
