"""The seeded synthetic workloads match the recipe the benchmarks and the
parity tests are quoted on: sizes, layout, the geometry each generator
promises, the bound on its ground-truth motion, the noise between source and
target, the scene's grid, and run-to-run determinism.  (CPU only.)"""
import math

import numpy as np
import pytest

import oracle
from paper_2512_04996_gb300 import synth


def _angle_deg(T):
    c = (np.trace(T[:3, :3]) - 1.0) / 2.0
    return math.degrees(math.acos(max(-1.0, min(1.0, c))))


def _check_layout(p, n):
    for a in (p.target, p.source):
        assert a.shape == (n, 4) and a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
        assert np.all(a[:, 3] == 0.0)
    R = p.T_gt[:3, :3]
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-12) and np.linalg.det(R) > 0
    assert np.array_equal(p.T_gt[3], [0.0, 0.0, 0.0, 1.0])


def _residual(p):
    """|T_gt s_i - q_i| per point (source and target in index correspondence)."""
    s = p.source[:, :3].astype(np.float64)
    return np.linalg.norm(s @ p.T_gt[:3, :3].T + p.T_gt[:3, 3] - p.target[:, :3], axis=1)


def test_sphere_plane_recipe():
    p = synth.sphere_plane()
    _check_layout(p, 4096)
    t = p.target[:, :3].astype(np.float64)
    assert np.abs(np.linalg.norm(t[:2048], axis=1) - 1.0).max() < 1e-6   # unit sphere
    assert np.all(t[2048:, 2] == -1.0)                                     # plane z = -1
    assert np.abs(t[2048:, :2]).max() <= 0.5
    assert _angle_deg(p.T_gt) <= 10.0 and np.linalg.norm(p.T_gt[:3, 3]) <= 0.05
    assert _residual(p).max() < 8 * 0.001                                  # N(0, 0.001^2) per axis
    assert (p.grid_divisions, p.iters) == (64, 30)


def test_bumpy_object_recipe():
    p = synth.bumpy_object()
    _check_layout(p, 40_000)
    t = p.target[:, :3].astype(np.float64)
    r = np.linalg.norm(t, axis=1)
    assert r.min() >= 0.9 - 1e-3 and r.max() <= 1.1 + 1e-3                # radial deviation <= 0.1
    assert r.max() - 1.0 > 0.05 or 1.0 - r.min() > 0.05                     # and it is used
    # acceptance rising linearly from 0.1 (south pole) to 1 (north pole):
    # expected north/south count ratio (0.1 + 0.9 * 3/4) / (0.1 + 0.9 / 4) = 2.385
    north, south = (t[:, 2] > 0).sum(), (t[:, 2] < 0).sum()
    assert 2.2 < north / south < 2.6
    assert _angle_deg(p.T_gt) <= 15.0 and np.linalg.norm(p.T_gt[:3, 3]) <= 0.1
    assert _residual(p).max() < 8 * 0.002
    assert (p.grid_divisions, p.iters) == (128, 50)


def test_depth_scene_recipe():
    p = synth.depth_scene()
    _check_layout(p, 226_000)
    assert p.voxel_size == 0.02 and p.iters == 30
    # target in camera 1's frame, depth clipped to [0.5, 5] m; the source's
    # depth carries sigma = 0.002 z^2 of noise after the clip
    z = p.target[:, 2]
    assert z.min() >= 0.5 and z.max() <= 5.0
    zs = p.source[:, 2]
    assert zs.min() >= 0.5 - 0.2 and zs.max() <= 5.0 + 0.2
    assert _angle_deg(p.T_gt) <= 5.0 and np.linalg.norm(p.T_gt[:3, 3]) <= 0.1
    # the benchmark's grid: 2 cm voxels over the target's box
    g = oracle.fit_grid(p.target, p.voxel_size, p.grid_divisions)
    assert tuple(g.dims) == (280, 177, 220) and int(np.prod(g.dims)) == 10_903_200


def test_batched_pairs_recipe_on_the_first_pairs():
    ps = synth.batched_pairs(n_pairs=6)
    assert len(ps) == 6
    for k, p in enumerate(ps):
        n = p.target.shape[0]
        assert 2000 <= n <= 64000
        _check_layout(p, n)
        assert ("sphere" in p.name) == (k % 2 == 0) and ("bumpy" in p.name) == (k % 2 == 1)
        assert _angle_deg(p.T_gt) <= 15.0 and np.linalg.norm(p.T_gt[:3, 3]) <= 0.2
        assert p.iters == 40
    # the first pairs of the full workload are these pairs
    assert [p.name for p in synth.batched_pairs(n_pairs=3)] == [p.name for p in ps[:3]]


@pytest.mark.parametrize("make", [synth.sphere_plane, lambda: synth.bumpy_object(n=5000), synth.depth_scene])
def test_generators_are_deterministic(make):
    a, b = make(), make()
    assert np.array_equal(a.target, b.target) and np.array_equal(a.source, b.source)
    assert np.array_equal(a.T_gt, b.T_gt)
