"""End-to-end sanity pins of the oracle's ICP loop.  The localised NNS is an
approximation, so the full loop has no exact closed form ("parity unpinned
against ground truth"); these tests check what must hold anyway."""
import json
import os

import numpy as np

import oracle


def _pose_error(T, T_gt):
    E = T @ np.linalg.inv(T_gt)
    ang = np.arccos(np.clip((np.trace(E[:3, :3]) - 1.0) / 2.0, -1.0, 1.0))
    return ang, np.linalg.norm(E[:3, 3])


def test_sphere_plane_converges_to_ground_truth(pairs):
    p = pairs(1)
    g = oracle.fit_grid(p.target, p.voxel_size, p.grid_divisions)
    st, T, it, hist = oracle.register(g, 10, p.target, p.source, np.eye(4), max_iters=30, eps=0.0)
    assert st == 0 and it == 30
    ang, tr = _pose_error(T, p.T_gt)
    assert ang < np.radians(0.05) and tr < 2e-3
    # residual falls to the noise floor: sigma * sqrt(3) per point, plus the
    # target's own sampling gap
    assert hist[-1] < hist[0] / 4
    assert hist[-1] < 0.01


def test_noise_free_identity_is_a_fixed_point(pairs):
    p = pairs(1)
    g = oracle.fit_grid(p.target, p.voxel_size, p.grid_divisions)
    st, T, it, hist = oracle.register(g, 10, p.target, p.target, np.eye(4), max_iters=3, eps=0.0)
    assert st == 0 and np.abs(T - np.eye(4)).max() < 1e-12
    assert np.all(hist == 0.0)


def test_early_stop_rule():
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")) as f:
        par = json.load(f)
    from paper_2512_04996_gb300 import synth
    p = synth.sphere_plane(seed=77, n=2000)
    g = oracle.fit_grid(p.target, 0.0, 64)
    st, T, it, hist = oracle.register(g, par["dilation_layers"], p.target, p.source, np.eye(4),
                                      max_iters=par["max_iters"], eps=par["rmse_eps"])
    assert st == 0 and 2 <= it < par["max_iters"]
    assert abs(hist[it - 1] - hist[it - 2]) < par["rmse_eps"]
    assert np.all(np.abs(np.diff(hist[: it - 1])) >= par["rmse_eps"])


def test_degenerate_source_reports_status():
    tgt = np.zeros((100, 4), np.float32)
    tgt[:, 0] = np.linspace(0, 1, 100)                      # points on a line
    g = oracle.fit_grid(tgt, 0.0, 16)
    st, T, it, hist = oracle.register(g, 4, tgt, tgt, np.eye(4), max_iters=5, eps=0.0)
    assert st == oracle.ERR_DEGENERATE and it == 0
    assert np.array_equal(T, np.eye(4))
