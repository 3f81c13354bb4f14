"""Pins of the oracle's dilation (Alg. 3) against a hand case and a brute-force
closed form.

The L synchronous rounds of Alg. 3 reach exactly the voxels within Manhattan
distance L of an occupied voxel (breadth-first search on a box grid, where
every monotone lattice path stays inside the box), and the min-root tie-break
keeps, among the occupied voxels at that minimum distance, the one with the
smallest linear index.  The brute force below computes that definition
directly, over all pairs of voxels."""
import numpy as np
import pytest

import oracle


def _off_from_occupancy(occ):
    counts = occ.astype(np.uint32)
    return np.concatenate([[0], np.cumsum(counts)]).astype(np.uint32)


def _brute_closed_form(dims, occ, L):
    nx, ny, nz = dims
    V = nx * ny * nz
    v = np.arange(V)
    xyz = np.stack([v % nx, (v // nx) % ny, v // (nx * ny)], axis=1)
    occ_idx = np.flatnonzero(occ)
    root = np.full(V, -1, np.int32)
    ring = np.full(V, 255, np.uint8)
    if occ_idx.size == 0:
        return root, ring
    d = np.abs(xyz[:, None, :] - xyz[None, occ_idx, :]).sum(axis=2)   # (V, n_occ) Manhattan
    dmin = d.min(axis=1)
    # smallest linear index among the occupied voxels at the minimum distance
    cand = np.where(d == dmin[:, None], occ_idx[None, :], np.iinfo(np.int64).max)
    rmin = cand.min(axis=1)
    lab = dmin <= L
    root[lab] = rmin[lab]
    ring[lab] = dmin[lab]
    return root, ring


def test_dilation_hand_case_row():
    # 9x1x1 row, occupied at x = 2 and x = 6, L = 3.  x = 4 is equidistant
    # (2 steps) from both and takes the smaller root, 2.
    occ = np.zeros(9, bool)
    occ[[2, 6]] = True
    g = oracle.explicit_grid((0, 0, 0), 1.0, (9, 1, 1))
    root, ring = oracle.dilate(g, _off_from_occupancy(occ), 3)
    assert root.tolist() == [2, 2, 2, 2, 2, 6, 6, 6, 6]
    assert ring.tolist() == [2, 1, 0, 1, 2, 1, 0, 1, 2]
    root, ring = oracle.dilate(g, _off_from_occupancy(occ), 1)
    assert root.tolist() == [-1, 2, 2, 2, -1, 6, 6, 6, -1]
    assert ring.tolist() == [255, 1, 0, 1, 255, 1, 0, 1, 255]


def test_dilation_hand_case_plane_tie():
    # 3x3x1 grid, occupied corners (0,0) and (2,2): the anti-diagonal voxels
    # (2,0), (1,1), (0,2) are 2 steps from both corners and keep root 0.
    occ = np.zeros(9, bool)
    occ[[0, 8]] = True
    g = oracle.explicit_grid((0, 0, 0), 1.0, (3, 3, 1))
    root, ring = oracle.dilate(g, _off_from_occupancy(occ), 5)
    assert root.tolist() == [0, 0, 0, 0, 0, 8, 0, 8, 8]
    assert ring.tolist() == [0, 1, 2, 1, 2, 1, 2, 1, 0]


@pytest.mark.parametrize("seed", range(8))
def test_dilation_equals_closed_form(seed):
    rng = np.random.default_rng(100 + seed)
    dims = tuple(int(v) for v in rng.integers(1, 13, 3))
    V = dims[0] * dims[1] * dims[2]
    occ = rng.uniform(size=V) < rng.choice([0.0, 0.005, 0.02, 0.1, 0.5])
    L = int(rng.integers(0, 8))
    g = oracle.explicit_grid((0, 0, 0), 1.0, dims)
    root, ring = oracle.dilate(g, _off_from_occupancy(occ), L)
    want_root, want_ring = _brute_closed_form(dims, occ, L)
    assert np.array_equal(root, want_root)
    assert np.array_equal(ring, want_ring)


def test_dilation_invariants(pairs):
    p = pairs(1)
    g = oracle.fit_grid(p.target, p.voxel_size, p.grid_divisions)
    b = oracle.build_grid(g, p.target, 10)
    occ = np.diff(b["off"].astype(np.int64)) > 0
    root, ring = b["root"], b["ring"]
    nx, ny, nz = g.dims
    # ring 0 exactly on occupied voxels, which are their own roots
    assert np.array_equal(ring == 0, occ)
    assert np.array_equal(root[occ], np.flatnonzero(occ).astype(np.int32))
    lab = root >= 0
    assert np.array_equal(lab, ring <= 10)
    # every root is occupied
    assert occ[root[lab]].all()
    # ring is 1-Lipschitz across labelled face neighbours
    r = ring.reshape(nz, ny, nx).astype(np.int32)
    lb = lab.reshape(nz, ny, nx)
    for ax in range(3):
        a = np.moveaxis(r, ax, 0)
        m = np.moveaxis(lb, ax, 0)
        both = m[1:] & m[:-1]
        assert (np.abs(a[1:] - a[:-1])[both] <= 1).all()
    # the ring equals the Manhattan distance to the root
    v = np.flatnonzero(lab)
    rv = root[lab].astype(np.int64)
    dist = (np.abs(v % nx - rv % nx) + np.abs((v // nx) % ny - (rv // nx) % ny)
            + np.abs(v // (nx * ny) - rv // (nx * ny)))
    assert np.array_equal(dist, ring[lab].astype(np.int64))


def test_dilation_zero_layers_keeps_only_occupied():
    rng = np.random.default_rng(3)
    occ = rng.uniform(size=6 * 7 * 8) < 0.1
    g = oracle.explicit_grid((0, 0, 0), 1.0, (6, 7, 8))
    root, ring = oracle.dilate(g, _off_from_occupancy(occ), 0)
    assert np.array_equal(root >= 0, occ)
    assert (ring[occ] == 0).all() and (ring[~occ] == 255).all()


def test_dilation_empty_grid():
    g = oracle.explicit_grid((0, 0, 0), 1.0, (5, 4, 3))
    root, ring = oracle.dilate(g, np.zeros(61, np.uint32), 10)
    assert (root == -1).all() and (ring == 255).all()
