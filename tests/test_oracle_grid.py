"""Pins of the oracle's grid build (Alg. 1 and Alg. 2) against hand cases,
closed forms and numpy library routines -- never against the oracle itself."""
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cloud(rng, n, lo=-1.0, hi=1.0):
    p = np.zeros((n, 4), np.float32)
    p[:, :3] = rng.uniform(lo, hi, (n, 3)).astype(np.float32)
    return p


# --- Quantize + Concat -------------------------------------------------------
def test_quantize_hand_cases():
    # origin 0, h = 0.5 (inv_h = 2 exactly), dims (4, 3, 2): key = x + 4*(y + 3*z)
    g = oracle.explicit_grid((0.0, 0.0, 0.0), 0.5, (4, 3, 2))
    assert g.inv_h == 2.0
    assert oracle.voxel_key(g, 0.0, 0.0, 0.0) == 0
    assert oracle.voxel_key(g, 0.5, 0.0, 0.0) == 1           # on the x face: upper voxel
    assert oracle.voxel_key(g, 0.49999997, 0.0, 0.0) == 0
    assert oracle.voxel_key(g, 1.2, 1.0, 0.6) == 2 + 4 * (2 + 3 * 1)
    assert oracle.voxel_key(g, 1.99, 1.49, 0.99) == 3 + 4 * (2 + 3 * 1)   # last voxel = V-1
    assert oracle.voxel_key(g, 2.0, 0.0, 0.0) == -1          # s == dims: outside
    assert oracle.voxel_key(g, 0.0, 1.5, 0.0) == -1
    assert oracle.voxel_key(g, 0.0, 0.0, 1.0) == -1
    assert oracle.voxel_key(g, -1e-7, 0.0, 0.0) == -1        # below the origin
    assert oracle.voxel_key(g, float("nan"), 0.0, 0.0) == -1
    assert oracle.voxel_key(g, 0.0, float("inf"), 0.0) == -1
    assert oracle.voxel_key(g, 0.0, 0.0, float("-inf")) == -1


def test_quantize_matches_float32_definition():
    """key from numpy float32 ops in the same order: d = p - o, s = d * inv_h."""
    rng = np.random.default_rng(1)
    pts = _cloud(rng, 5000, -0.2, 1.3)
    g = oracle.explicit_grid((0.05, -0.1, 0.0), 0.037, (31, 29, 33))
    o = np.array(g.origin, np.float32)
    s = (pts[:, :3] - o) * np.float32(g.inv_h)
    dims = np.array(g.dims)
    inside = np.all((s >= 0) & (s < dims.astype(np.float32)), axis=1)
    i = np.floor(s).astype(np.int64)
    want = np.where(inside, i[:, 0] + dims[0] * (i[:, 1] + dims[1] * i[:, 2]), -1)
    assert np.array_equal(oracle.keys(g, pts), want.astype(np.int32))


def test_fit_grid_contains_every_target_point(pairs):
    for k in (1, 2, 3):
        p = pairs(k)
        g = oracle.fit_grid(p.target, p.voxel_size, p.grid_divisions)
        t = p.target[:, :3]
        assert g.origin == tuple(float(v) for v in t.min(axis=0))
        ext = t.max(axis=0) - t.min(axis=0)
        h = np.float32(p.voxel_size) if p.voxel_size else np.float32(ext.max()) / np.float32(p.grid_divisions)
        assert np.float32(g.h) == h
        assert np.float32(g.inv_h) == np.float32(1.0 / np.float64(h))
        assert g.dims == tuple(int(v) for v in np.floor(ext * np.float32(g.inv_h)).astype(np.int64) + 1)
        keys = oracle.keys(g, p.target)
        assert (keys >= 0).all()
        assert keys.max() < g.n_voxels


def test_fit_grid_single_point():
    p = np.array([[0.25, -3.0, 7.5, 0.0]], np.float32)
    g = oracle.fit_grid(p, 0.0, 64)
    assert g.dims == (1, 1, 1) and g.h == 1.0
    assert oracle.keys(g, p)[0] == 0


# --- VOH / MOC / VDMA --------------------------------------------------------
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_histogram_offsets_csr_invariants(seed):
    rng = np.random.default_rng(seed)
    n = 3000
    pts = _cloud(rng, n)
    pts[::7, :3] = pts[0, :3]                    # one crowded voxel
    g = oracle.explicit_grid((-0.9, -1.0, -1.0), 0.1, (17, 21, 19))   # some points outside
    keys = oracle.keys(g, pts)
    V = g.n_voxels
    inside = keys >= 0
    assert 0 < inside.sum() < n

    counts = oracle.histogram(keys, V)
    assert np.array_equal(counts, np.bincount(keys[inside], minlength=V).astype(np.uint32))
    assert int(counts.sum()) == int(inside.sum())

    off = oracle.offsets(counts)
    assert off[0] == 0 and off[-1] == inside.sum()
    assert np.array_equal(off[1:], np.cumsum(counts, dtype=np.uint64).astype(np.uint32))

    ids = oracle.csr(keys, off)
    # Permutation of the inside points, grouped by key, ascending inside a segment:
    # exactly a stable sort of the inside points by key.
    want = np.flatnonzero(inside)[np.argsort(keys[inside], kind="stable")]
    assert np.array_equal(ids, want.astype(np.int32))
    for v in np.flatnonzero(counts)[:50]:
        seg = ids[off[v]:off[v + 1]]
        assert (keys[seg] == v).all() and (np.diff(seg) > 0).all()


def test_paper_moc_layout():
    """Alg. 1's CPU part reserves count+2 words per voxel (two header words), so
    its address of voxel v is the header-free offset plus 2v."""
    rng = np.random.default_rng(5)
    counts = rng.integers(0, 5, 1000).astype(np.uint32)
    counts[rng.uniform(size=1000) < 0.6] = 0
    off = oracle.offsets(counts)
    addr = oracle.paper_moc(counts)
    assert np.array_equal(addr.astype(np.int64), off[:-1].astype(np.int64) + 2 * np.arange(1000))


def test_paper_static_memory_pin():
    """Table 1 note 1: histogram + address offsets take 0.03125 MB at N = 4."""
    with open(os.path.join(GOLDEN, "paper_static_memory.json")) as f:
        gold = json.load(f)
    V = (2 ** gold["N"]) ** 3
    assert gold["voxels_per_axis"] ** 3 == V
    assert oracle.paper_static_bytes(V) / gold["megabyte"] == gold["static_megabytes"]


def test_build_grid_matches_steps(pairs):
    p = pairs(1)
    g = oracle.fit_grid(p.target, p.voxel_size, p.grid_divisions)
    b = oracle.build_grid(g, p.target, 10)
    keys = oracle.keys(g, p.target)
    assert np.array_equal(b["keys"], keys)
    assert np.array_equal(b["off"], oracle.offsets(oracle.histogram(keys, g.n_voxels)))
    assert np.array_equal(b["ids"], oracle.csr(keys, b["off"]))
    root, ring = oracle.dilate(g, b["off"], 10)
    assert np.array_equal(b["root"], root) and np.array_equal(b["ring"], ring)


def test_fit_grid_ignores_nan_coordinates():
    p = np.array([[np.nan, 0, 0, 0], [0.5, 1.0, -2.0, 0], [1.5, 0.0, 0.0, 0]], np.float32)
    g = oracle.fit_grid(p, 0.25, 0)
    assert g.origin == (0.5, 0.0, -2.0)
    assert g.dims == (5, 5, 9)
    with pytest.raises(ValueError):
        oracle.fit_grid(np.array([[np.nan, 0, 0, 0]], np.float32), 0.25, 0)
