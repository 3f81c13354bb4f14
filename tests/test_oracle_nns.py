"""Pins of the oracle's localised NNS (Alg. 4): brute force over the root
voxel's segment, exact brute-force global NN for the fallback, and the
single-voxel special case that reduces to exact nearest neighbours."""
import numpy as np
import pytest

import oracle


def _transform_f32(T, pts):
    """s_a = ((R_a0*x + R_a1*y) + R_a2*z) + t_a in float32, one rounding per op."""
    R = T[:3, :3].astype(np.float32)
    t = T[:3, 3].astype(np.float32)
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    out = np.empty((pts.shape[0], 3), np.float32)
    for a in range(3):
        acc = R[a, 0] * x
        acc = acc + R[a, 1] * y
        acc = acc + R[a, 2] * z
        out[:, a] = acc + t[a]
    return out


def _d2_f32(s, q):
    d = s[:, None, :] - q[None, :, :3]
    acc = d[..., 0] * d[..., 0]
    acc = acc + d[..., 1] * d[..., 1]
    return acc + d[..., 2] * d[..., 2]


def _argmin_ties_low(d2, idx):
    """Strict minimum, ties to the smaller index."""
    order = np.lexsort((idx, d2))
    return idx[order[0]], d2[order[0]]


def _rigid(rng, deg, trans):
    from paper_2512_04996_gb300.synth import random_rigid
    return random_rigid(rng, deg, trans)


def test_correspond_local_and_fallback_by_brute_force(pairs):
    p = pairs(1)
    rng = np.random.default_rng(7)
    g = oracle.fit_grid(p.target, p.voxel_size, p.grid_divisions)
    b = oracle.build_grid(g, p.target, 3)          # small L: many fallbacks
    T = _rigid(rng, 20.0, 0.3)
    src = p.source[:1500]
    nn, d2, fb = oracle.correspond(g, b, p.target, src, T)
    assert 50 < fb.sum() < 1450
    s = _transform_f32(T, src)
    keys = oracle.keys(g, np.column_stack([s, np.zeros(len(s), np.float32)]))
    for i in range(0, len(src), 3):
        v = keys[i]
        r = b["root"][v] if v >= 0 else -1
        if r >= 0:
            seg = b["ids"][b["off"][r]:b["off"][r + 1]]
            assert not fb[i]
        else:
            seg = np.arange(p.target.shape[0])
            assert fb[i]
        dd = _d2_f32(s[i:i + 1], p.target[seg])[0]
        j, dj = _argmin_ties_low(dd, seg)
        assert nn[i] == j and d2[i] == dj


def test_single_voxel_grid_is_exact_nn():
    """With one voxel holding every target point, the local search is the
    exact nearest-neighbour search."""
    rng = np.random.default_rng(11)
    tgt = np.zeros((700, 4), np.float32)
    tgt[:, :3] = rng.uniform(-1, 1, (700, 3))
    src = np.zeros((300, 4), np.float32)
    src[:, :3] = rng.uniform(-1.2, 1.2, (300, 3))
    g = oracle.explicit_grid((-1.0, -1.0, -1.0), 2.0, (1, 1, 1))
    b = oracle.build_grid(g, tgt, 0)
    T = np.eye(4)
    nn, d2, fb = oracle.correspond(g, b, tgt, src, T)
    s = _transform_f32(T, src)
    dd = _d2_f32(s, tgt)
    inside = oracle.keys(g, src) >= 0
    assert (fb == ~inside).all()
    for i in range(300):
        j, dj = _argmin_ties_low(dd[i], np.arange(700))
        assert nn[i] == j and d2[i] == dj


def test_tie_goes_to_smaller_index():
    tgt = np.array([[0, 0, 5, 0], [1, 0, 0, 0], [-1, 0, 0, 0], [0, 1, 0, 0]], np.float32)
    src = np.zeros((1, 4), np.float32)                # equidistant (d2 = 1) from rows 1, 2, 3
    g = oracle.explicit_grid((-10, -10, -10), 100.0, (1, 1, 1))
    b = oracle.build_grid(g, tgt, 0)
    nn, d2, fb = oracle.correspond(g, b, tgt, src, np.eye(4))
    assert nn[0] == 1 and d2[0] == 1.0 and not fb[0]


def test_outside_source_takes_global_search():
    rng = np.random.default_rng(2)
    tgt = np.zeros((200, 4), np.float32)
    tgt[:, :3] = rng.uniform(0, 1, (200, 3))
    g = oracle.explicit_grid((0, 0, 0), 0.25, (4, 4, 4))
    b = oracle.build_grid(g, tgt, 10)
    src = np.array([[5, 5, 5, 0], [-1, 0.5, 0.5, 0], [np.nan, 0, 0, 0]], np.float32)
    nn, d2, fb = oracle.correspond(g, b, tgt, src, np.eye(4))
    assert fb.all()
    dd = _d2_f32(src[:2, :3], tgt)
    for i in range(2):
        j, dj = _argmin_ties_low(dd[i], np.arange(200))
        assert nn[i] == j and d2[i] == dj


def test_reduce_matches_two_pass_definition(pairs):
    p = pairs(1)
    rng = np.random.default_rng(4)
    T = _rigid(rng, 5.0, 0.05)
    nn = rng.integers(0, p.target.shape[0], p.source.shape[0]).astype(np.int32)
    pbar, qbar, H, rmse = oracle.reduce(p.target, p.source, T, nn)
    s = _transform_f32(T, p.source).astype(np.float64)
    q = p.target[nn, :3].astype(np.float64)
    assert np.allclose(pbar, s.mean(0), rtol=0, atol=1e-14)
    assert np.allclose(qbar, q.mean(0), rtol=0, atol=1e-14)
    Hw = (s - s.mean(0)).T @ (q - q.mean(0))
    assert np.allclose(H, Hw, rtol=1e-12, atol=1e-12)
    assert abs(rmse - np.sqrt(((s - q) ** 2).sum(1).mean())) < 1e-13


def test_nan_target_never_beats_a_number():
    """A target point with a NaN coordinate has a NaN distance; the search
    orders NaN after every number, wherever the NaN point sits in the list."""
    tgt = np.array([[np.nan, 0, 0, 0], [3, 0, 0, 0], [2, 0, 0, 0], [np.nan, 1, 1, 0]], np.float32)
    src = np.zeros((1, 4), np.float32)
    g = oracle.explicit_grid((5, 5, 5), 1.0, (1, 1, 1))      # source outside: global search
    b = oracle.build_grid(g, tgt, 0)
    nn, d2, fb = oracle.correspond(g, b, tgt, src, np.eye(4))
    assert fb[0] and nn[0] == 2 and d2[0] == 4.0
