"""GPU NNS (Alg. 4) against the oracle: for every source point the same target
index and the same float squared distance (the tolerance allows another index
only when its squared distance is within 1e-6 relative), and the same set of
points taking the global search."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import assert_nn_equal, gpu_grid, oracle_grid_for, to_np, transform_f32
from paper_2512_04996_gb300.synth import random_rigid

pytestmark = pytest.mark.gpu


def _gpu_correspond(ctx, src, T):
    s = torch.from_numpy(np.ascontiguousarray(src)).cuda()
    pose = torch.from_numpy(np.ascontiguousarray(T, dtype=np.float64)).cuda()
    nn, d2, nf = ctx.correspond(s, pose)
    torch.cuda.synchronize()
    return to_np(nn), to_np(d2), int(to_np(nf)[0])


def _assert_nn_equal(nn, d2, rnn, rd2, target=None):
    assert_nn_equal(nn, d2, rnn, rd2)


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("which", ["identity", "ground_truth", "random"])
def test_correspond_matches_oracle(pairs, k, which):
    p = pairs(k)
    ctx, g = gpu_grid(p.target, L=10, voxel_size=p.voxel_size, divisions=p.grid_divisions)
    grid, ref = oracle_grid_for(g, p.target, 10)
    T = {"identity": np.eye(4), "ground_truth": p.T_gt,
         "random": random_rigid(np.random.default_rng(k), 25.0, 0.3)}[which]
    nn, d2, nf = _gpu_correspond(ctx, p.source, T)
    rnn, rd2, rfb = oracle.correspond(grid, ref, p.target, p.source, T)
    assert nf == int(rfb.sum())
    _assert_nn_equal(nn, d2, rnn, rd2, p.target)


@pytest.mark.parametrize("which", ["identity", "ground_truth"])
def test_correspond_scene_full(pairs, oracle_threads, which):
    """The full 226k-point scene: every source point's neighbour against the
    oracle's, and the global-search count."""
    p = pairs(3)
    ctx, g = gpu_grid(p.target, L=10, voxel_size=p.voxel_size)
    grid, ref = oracle_grid_for(g, p.target, 10)
    T = p.T_gt if which == "ground_truth" else np.eye(4)
    nn, d2, nf = _gpu_correspond(ctx, p.source, T)
    rnn, rd2, rfb = oracle.correspond(grid, ref, p.target, p.source, T)
    _assert_nn_equal(nn, d2, rnn, rd2, p.target)
    assert nf == int(rfb.sum()) and 0 < nf < p.source.shape[0]
    # the fallback set is the points outside the grid or in an unlabelled voxel
    keys = oracle.keys(grid, transform_f32(T, p.source))
    assert np.array_equal(rfb, (keys < 0) | (ref["root"][np.maximum(keys, 0)] < 0))


def test_global_search_with_outside_targets_and_odd_sources():
    """Explicit grid: targets outside it are reachable only by the global
    search; sources outside, far away, NaN and infinite take it too."""
    rng = np.random.default_rng(5)
    tgt = np.zeros((3001, 4), np.float32)
    tgt[:, :3] = rng.uniform(-0.5, 1.5, (3001, 3))
    src = np.zeros((1000, 4), np.float32)
    src[:, :3] = rng.uniform(-1.0, 2.0, (1000, 3))
    src[0, :3] = [50.0, -40.0, 7.0]
    src[1, 0] = np.nan
    src[2, 1] = np.inf
    ctx, g = gpu_grid(tgt, L=2, voxel_size=0.1, origin=(0.0, 0.0, 0.0), dims=(10, 10, 10))
    grid, ref = oracle_grid_for(g, tgt, 2)
    nn, d2, nf = _gpu_correspond(ctx, src, np.eye(4))
    rnn, rd2, rfb = oracle.correspond(grid, ref, tgt, src, np.eye(4))
    assert nf == int(rfb.sum())
    _assert_nn_equal(nn, d2, rnn, rd2, tgt)
    assert nn[1] == 0 and np.isnan(d2[1])


def test_empty_voxels_everywhere_forces_global_search():
    """L = 0 and a pose far from the target: every point takes the global
    search, which must still be exact."""
    rng = np.random.default_rng(6)
    tgt = np.zeros((20000, 4), np.float32)
    tgt[:, :3] = rng.standard_normal((20000, 3))
    src = np.zeros((4000, 4), np.float32)
    src[:, :3] = rng.standard_normal((4000, 3))
    ctx, g = gpu_grid(tgt, L=0, divisions=256)
    grid, ref = oracle_grid_for(g, tgt, 0)
    T = np.eye(4)
    T[:3, 3] = [0.003, -0.002, 0.001]
    nn, d2, nf = _gpu_correspond(ctx, src, T)
    rnn, rd2, rfb = oracle.correspond(grid, ref, tgt, src, T)
    assert nf == int(rfb.sum()) and nf > 3000
    _assert_nn_equal(nn, d2, rnn, rd2, tgt)


def test_nn_ties_go_to_smaller_index():
    tgt = np.zeros((64, 4), np.float32)
    tgt[:32, 0] = 1.0          # 32 copies of the same point ...
    tgt[32:, 0] = -1.0         # ... and 32 mirror images, all at distance 1 from 0
    src = np.zeros((40, 4), np.float32)
    for L, origin, dims in ((10, (-1.0, -1.0, -1.0), (3, 3, 3)), (0, (5.0, 5.0, 5.0), (2, 2, 2))):
        ctx, g = gpu_grid(tgt, L=L, voxel_size=1.0, origin=origin, dims=dims)
        nn, d2, nf = _gpu_correspond(ctx, src, np.eye(4))
        grid, ref = oracle_grid_for(g, tgt, L)
        rnn, rd2, rfb = oracle.correspond(grid, ref, tgt, src, np.eye(4))
        assert np.array_equal(nn, rnn)


def test_searches_read_only_the_offsets_the_build_writes(pairs):
    """The build writes only part of the offsets array (occupied voxels, the
    entries just past them, every 32nd one); a grid view completes it.  Fill
    the array with one cloud's offsets, rebuild the same grid with another
    cloud (other occupied voxels) and search without a view in between: any
    read of an entry the second build did not write would see the first
    cloud's offsets and miss the oracle's neighbours."""
    p = pairs(2)
    ctx, g = gpu_grid(p.target, L=10, voxel_size=p.voxel_size, divisions=p.grid_divisions)
    rng = np.random.default_rng(12)
    tgt_b = p.target[rng.random(p.target.shape[0]) < 0.6].copy()
    tgt_b[:, 0] += np.float32(0.37 * g["voxel_size"])
    tgt_b = np.ascontiguousarray(tgt_b)
    ctx2, g2 = gpu_grid(tgt_b, L=10, origin=g["origin"], voxel_size=g["voxel_size"], dims=g["dims"])
    assert not np.array_equal(g2["occupancy"], g["occupancy"])
    # the first cloud's dense offsets in ctx2's array, then the second build
    ctx2.build_grid(g["_target"])
    ctx2.get_grid()
    ctx2.build_grid(g2["_target"])
    ctx2.dilate(10)
    grid, ref = oracle_grid_for(g2, tgt_b, 10)
    for T in (np.eye(4), p.T_gt):
        nn, d2, nf = _gpu_correspond(ctx2, p.source, T)
        rnn, rd2, rfb = oracle.correspond(grid, ref, tgt_b, p.source, T)
        assert nf == int(rfb.sum())
        _assert_nn_equal(nn, d2, rnn, rd2, tgt_b)
    # and the completed array is the oracle's
    assert np.array_equal(to_np(ctx2.get_grid()["offsets"]), ref["off"])
