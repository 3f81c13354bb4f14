"""The sparse (hashed) grid (VICP_FLAG_SPARSE_GRID) against the oracle.

Its tables are mapped back to dense per-voxel arrays here and compared bit
for bit: the occupied-voxel table's keys and counts with the oracle's
histogram, every voxel's CSR segment with the oracle's as a set, the
labelled-segment table (a label mask and a slice of the root array per 32
voxels along x) as labelled voxels, roots and rings (the Manhattan distance
between a voxel and its root) with the oracle's dilation.  Searches and
registrations must equal the oracle's at the usual tolerances -- and the
dense grid's results bit for bit, since both grids feed the same search and
reduction the same candidates in the same order.  Also: rebuilding with
another cloud in the same context, the long-L path, degenerate clouds, and
the memory it saves on the scene."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import assert_nn_equal, context, rot_err, to_np, transform_f32
from paper_2512_04996_gb300.synth import random_rigid

pytestmark = pytest.mark.gpu

EMPTY = 0xFFFFFFFF


def _sparse_flags(extra=0):
    from paper_2512_04996_gb300 import vicp
    return vicp.VICP_FLAG_SPARSE_GRID | extra


def _sparse_grid(target, L=10, **kw):
    ctx = context(L=L, flags=_sparse_flags(kw.pop("flags", 0)), **kw)
    t = torch.from_numpy(np.ascontiguousarray(target)).cuda()
    ctx.build_grid(t)
    ctx.dilate(L)
    g = {k: to_np(v) for k, v in ctx.get_sparse_grid().items()}
    g["_target"] = t
    return ctx, g


def _coords(keys, dims):
    keys = keys.astype(np.int64)
    nx, ny = dims[0], dims[1]
    return np.stack([keys % nx, (keys // nx) % ny, keys // (nx * ny)], axis=1)


def assert_sparse_equal(g, ref, target):
    """The sparse tables mapped to dense arrays, against the oracle's build."""
    V = int(g["n_voxels"])
    assert np.array_equal(g["keys"], ref["keys"])
    assert g["n_stored"] == int(ref["off"][-1])
    # occupied voxels: keys, counts and segments
    okeys = g["occupied_keys"]
    occ_slots = np.flatnonzero(okeys != EMPTY)
    vox = okeys[occ_slots].astype(np.int64)
    counts = np.diff(ref["off"].astype(np.int64))
    assert np.array_equal(np.sort(vox), np.flatnonzero(counts))
    off = g["occupied_offsets"].astype(np.int64)
    a, b = off[occ_slots], off[occ_slots + 1]
    assert np.array_equal(b - a, counts[vox])
    assert int(off[-1]) == g["n_stored"]
    # the segments partition the store, in slot order
    order = np.argsort(a, kind="stable")
    a_s, b_s = a[order], b[order]
    assert a_s[0] == 0 and np.array_equal(a_s[1:], b_s[:-1]) and b_s[-1] == g["n_stored"]
    store_vox = np.repeat(vox[order], b_s - a_s)
    ids = g["ids"]
    assert np.array_equal(ids[np.lexsort((ids, store_vox))], ref["ids"])
    pts = g["csr_points"]
    assert np.array_equal(pts[:, :3], target[ids, :3])
    assert np.array_equal(pts[:, 3].view(np.int32), ids)
    bits = np.unpackbits(g["occupancy"].view(np.uint8), bitorder="little")[:V]
    assert np.array_equal(bits.astype(bool), counts > 0)
    # labelled voxels: exactly the oracle's, with its roots and rings.  The
    # table holds row segments (32 voxels along x): each entry's mask names
    # its labelled voxels and its base the first of their roots, which
    # follow in the order of x
    lkeys = g["labelled_keys"]
    lab = np.flatnonzero(lkeys != EMPTY)
    assert g["labelled_segment_count"] == lab.shape[0]
    nx, ny = g["dims"][0], g["dims"][1]
    nxb = (nx + 31) // 32
    sid = lkeys[lab].astype(np.int64)
    seg = g["labelled_segments"][lab].astype(np.int64)
    bits = ((seg[:, :1] >> np.arange(32)) & 1).astype(bool)          # [segments, 32]
    assert bits.any(axis=1).all()
    s_idx, bit = np.nonzero(bits)
    x = 32 * (sid[s_idx] % nxb) + bit
    assert (x < nx).all()
    lv = x + nx * (sid[s_idx] // nxb)                                 # row = y + ny z
    rank = np.cumsum(bits, axis=1)[s_idx, bit] - 1
    ridx = seg[s_idx, 1] + rank
    want = np.flatnonzero(ref["root"] >= 0)
    assert g["labelled_voxels"] == want.shape[0]
    assert np.array_equal(np.sort(lv), want)
    # the roots array is covered exactly once, segment by segment
    assert np.array_equal(np.sort(ridx), np.arange(g["labelled_voxels"]))
    root = g["labelled_root"][ridx]
    assert np.array_equal(root, ref["root"][lv])
    ring = np.abs(_coords(lv, g["dims"]) - _coords(root, g["dims"])).sum(axis=1)
    assert np.array_equal(ring, ref["ring"][lv].astype(np.int64))


def _oracle_for(g, target, L):
    grid = oracle.Grid(g["origin"], g["voxel_size"], g["inv_voxel_size"], g["dims"])
    return grid, oracle.build_grid(grid, target, L)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_sparse_grid_equals_oracle(pairs, oracle_threads, k):
    p = pairs(k)
    ctx, g = _sparse_grid(p.target, L=10, voxel_size=p.voxel_size, divisions=p.grid_divisions)
    grid, ref = _oracle_for(g, p.target, 10)
    assert_sparse_equal(g, ref, p.target)


@pytest.mark.parametrize("L", [0, 1, 5, 15, 16, 23])
def test_sparse_grid_dilation_depths(pairs, L):
    p = pairs(2)
    ctx, g = _sparse_grid(p.target, L=L, voxel_size=p.voxel_size, divisions=p.grid_divisions)
    grid, ref = _oracle_for(g, p.target, L)
    assert_sparse_equal(g, ref, p.target)


def _correspond(ctx, src, T):
    s = torch.from_numpy(np.ascontiguousarray(src)).cuda()
    pose = torch.from_numpy(np.ascontiguousarray(T, dtype=np.float64)).cuda()
    nn, d2, nf = ctx.correspond(s, pose)
    torch.cuda.synchronize()
    return to_np(nn), to_np(d2), int(to_np(nf)[0])


@pytest.mark.parametrize("k", [1, 2, 3])
def test_sparse_correspond_equals_oracle_and_dense(pairs, oracle_threads, k):
    p = pairs(k)
    ctx, g = _sparse_grid(p.target, L=10, voxel_size=p.voxel_size, divisions=p.grid_divisions)
    grid, ref = _oracle_for(g, p.target, 10)
    dense = context(L=10, voxel_size=p.voxel_size, divisions=p.grid_divisions)
    dense.build_grid(g["_target"])
    dense.dilate(10)
    for T in (np.eye(4), p.T_gt, random_rigid(np.random.default_rng(k), 20.0, 0.2)):
        nn, d2, nf = _correspond(ctx, p.source, T)
        rnn, rd2, rfb = oracle.correspond(grid, ref, p.target, p.source, T)
        assert_nn_equal(nn, d2, rnn, rd2)
        assert nf == int(rfb.sum())
        dnn, dd2, dnf = _correspond(dense, p.source, T)
        assert np.array_equal(nn, dnn) and np.array_equal(d2.view(np.uint32), dd2.view(np.uint32)) and nf == dnf


@pytest.mark.parametrize("k", [1, 2])
def test_sparse_register_matches_oracle(pairs, k):
    p = pairs(k)
    ctx = context(L=10, voxel_size=p.voxel_size, divisions=p.grid_divisions, max_iters=p.iters, eps=0.0,
                  flags=_sparse_flags())
    st, T, it, rm = ctx.register(torch.from_numpy(p.source).cuda(), torch.from_numpy(p.target).cuda())
    assert st == 0 and it == p.iters
    grid = oracle.fit_grid(p.target, p.voxel_size, p.grid_divisions)
    rst, R, rit, hist = oracle.register(grid, 10, p.target, p.source, np.eye(4), max_iters=p.iters, eps=0.0)
    assert rst == 0 and rit == it
    ext = float((p.target[:, :3].max(0) - p.target[:, :3].min(0)).max())
    assert rot_err(T, R) <= 1e-5 and np.linalg.norm(T[:3, 3] - R[:3, 3]) <= 1e-5 * ext
    assert abs(rm - hist[-1]) <= 1e-7 * hist[-1]


def test_sparse_scene_registration_equals_dense_bit_for_bit(pairs):
    """The scene, grid rebuilt every iteration, 30 iterations: the sparse and
    the dense grid give the same pose and RMSE bit for bit."""
    from paper_2512_04996_gb300 import vicp
    p = pairs(3)
    out = []
    for flags in (0, vicp.VICP_FLAG_SPARSE_GRID):
        ctx = context(L=10, voxel_size=p.voxel_size, max_iters=30, eps=0.0,
                      flags=flags | vicp.VICP_FLAG_KEEP_GRID | vicp.VICP_FLAG_REBUILD_EACH_ITER)
        out.append(ctx.register(torch.from_numpy(p.source).cuda(), torch.from_numpy(p.target).cuda()))
    assert out[0][0] == out[1][0] == 0 and out[0][2] == out[1][2] == 30
    assert np.array_equal(out[0][1], out[1][1]) and out[0][3] == out[1][3]


def test_sparse_rebuild_with_other_clouds_in_one_context(pairs):
    """Consecutive builds of different clouds (and grid sizes) in one
    context: every build's tables are the oracle's (the next build's tables
    are reset by the previous scatter and dilation)."""
    ctx = context(L=10, divisions=128, flags=_sparse_flags())
    for k in (2, 1, 2, 3, 1):
        p = pairs(k)
        ctx.build_grid(torch.from_numpy(p.target).cuda())
        ctx.dilate(10)
        g = {key: to_np(v) for key, v in ctx.get_sparse_grid().items()}
        grid, ref = _oracle_for(g, p.target, 10)
        assert_sparse_equal(g, ref, p.target)


def test_sparse_outside_targets_odd_sources_and_degenerate_clouds():
    rng = np.random.default_rng(5)
    tgt = np.zeros((3001, 4), np.float32)
    tgt[:, :3] = rng.uniform(-0.5, 1.5, (3001, 3))
    src = np.zeros((1000, 4), np.float32)
    src[:, :3] = rng.uniform(-1.0, 2.0, (1000, 3))
    src[0, :3] = [50.0, -40.0, 7.0]
    src[1, 0] = np.nan
    ctx, g = _sparse_grid(tgt, L=2, voxel_size=0.1, origin=(0.0, 0.0, 0.0), dims=(10, 10, 10))
    grid, ref = _oracle_for(g, tgt, 2)
    assert_sparse_equal(g, ref, tgt)
    nn, d2, nf = _correspond(ctx, src, np.eye(4))
    rnn, rd2, rfb = oracle.correspond(grid, ref, tgt, src, np.eye(4))
    assert nf == int(rfb.sum())
    assert_nn_equal(nn, d2, rnn, rd2)
    # one point; all points in one voxel
    for cloud in (tgt[:1].copy(), np.tile(np.array([[0.2, -0.1, 0.4, 0.0]], np.float32), (300, 1))):
        ctx, g = _sparse_grid(cloud, L=3, divisions=16)
        grid, ref = _oracle_for(g, cloud, 3)
        assert_sparse_equal(g, ref, cloud)


def test_sparse_grid_memory_on_the_scene(pairs):
    """The scene's peak device bytes: the sparse grid needs far less than the
    dense grid (its per-voxel arrays are replaced by the two tables)."""
    from paper_2512_04996_gb300 import vicp
    p = pairs(3)
    peak = {}
    for name, flags in (("dense", 0), ("sparse", vicp.VICP_FLAG_SPARSE_GRID)):
        ctx = context(L=10, voxel_size=p.voxel_size, max_iters=2, eps=0.0, flags=flags)
        st, *_ = ctx.register(torch.from_numpy(p.source).cuda(), torch.from_numpy(p.target).cuda())
        assert st == 0
        rep = ctx.memory_report()
        peak[name] = rep["peak_bytes"]
        if name == "sparse":
            assert rep["labelled_voxels"] > 0 and rep["occupied_voxels"] > 0
    assert peak["sparse"] < 0.5 * peak["dense"], peak


def test_sparse_rejects_the_dense_views(pairs):
    from paper_2512_04996_gb300 import vicp
    p = pairs(1)
    ctx, g = _sparse_grid(p.target, L=10, divisions=64)
    with pytest.raises(vicp.VicpError) as e:
        ctx.get_grid()
    assert e.value.status == vicp.VICP_ERR_STATE
    with pytest.raises(vicp.VicpError) as e:
        ctx.fixed_build(g["_target"], 8)
    assert e.value.status == vicp.VICP_ERR_STATE
    dense = context(L=10, divisions=64)
    dense.build_grid(g["_target"])
    with pytest.raises(vicp.VicpError) as e:
        dense.get_sparse_grid()
    assert e.value.status == vicp.VICP_ERR_STATE


def test_sparse_kept_grid_reports_a_cloud_that_outgrows_the_table(pairs):
    """Under VICP_FLAG_KEEP_GRID the labelled-segment table keeps the size the
    first dilation found: a much larger cloud in the same grid is reported by
    the next synchronising call (VICP_ERR_STATE), and the dilation after that
    checks and grows the table again, giving the oracle's labels."""
    from paper_2512_04996_gb300 import vicp
    p = pairs(2)
    _, g0 = _sparse_grid(p.target, L=10, divisions=128)
    kw = dict(origin=g0["origin"], voxel_size=g0["voxel_size"], dims=g0["dims"])
    ctx = context(L=10, flags=_sparse_flags(vicp.VICP_FLAG_KEEP_GRID), **kw)
    small = np.ascontiguousarray(p.target[:50])
    ctx.build_grid(torch.from_numpy(small).cuda())
    ctx.dilate(10)
    assert ctx.sync() == 0
    big = torch.from_numpy(p.target).cuda()
    ctx.build_grid(big)
    ctx.dilate(10)                           # kept size: no check, too small
    assert ctx.sync() == vicp.VICP_ERR_STATE
    ctx.build_grid(big)
    ctx.dilate(10)                           # checked again: grown
    assert ctx.sync() == 0
    g = {key: to_np(v) for key, v in ctx.get_sparse_grid().items()}
    grid, ref = _oracle_for(g, p.target, 10)
    assert_sparse_equal(g, ref, p.target)
    ctx.build_grid(big)                      # and kept from here on
    ctx.dilate(10)
    assert ctx.sync() == 0


def test_sparse_histogram_with_more_slot_tiles_than_shared_memory_holds():
    """8.5M points on a 256^3 grid: the occupied-voxel table has 2^25 slots,
    2,048 scan tiles -- more than a block's shared-memory tile totals hold,
    so the histogram adds its tile totals per warp.  Keys, per-voxel counts,
    segments and the CSR store against the oracle's keys and histogram."""
    rng = np.random.default_rng(11)
    n = 8_500_000
    tgt = np.zeros((n, 4), np.float32)
    tgt[:, :3] = rng.uniform(0.0, 1.0, (n, 3))
    ctx, g = _sparse_grid(tgt, L=1, voxel_size=1.0 / 256, origin=(0.0, 0.0, 0.0), dims=(256, 256, 256))
    okeys = g["occupied_keys"]
    assert okeys.shape[0] == 1 << 25
    grid = oracle.Grid(g["origin"], g["voxel_size"], g["inv_voxel_size"], g["dims"])
    keys = oracle.keys(grid, tgt)
    assert np.array_equal(g["keys"], keys)
    V = int(np.prod(g["dims"]))
    counts = np.bincount(keys[keys >= 0], minlength=V)
    occ_slots = np.flatnonzero(okeys != EMPTY)
    vox = okeys[occ_slots].astype(np.int64)
    assert np.array_equal(np.sort(vox), np.flatnonzero(counts))
    off = g["occupied_offsets"].astype(np.int64)
    a, b = off[occ_slots], off[occ_slots + 1]
    assert np.array_equal(b - a, counts[vox])
    assert int(off[-1]) == g["n_stored"] == int((keys >= 0).sum())
    order = np.argsort(a, kind="stable")
    a_s, b_s = a[order], b[order]
    assert a_s[0] == 0 and np.array_equal(a_s[1:], b_s[:-1])
    store_vox = np.repeat(vox[order], b_s - a_s)
    ids = g["ids"]
    assert np.array_equal(keys[ids], store_vox)
    assert np.array_equal(np.sort(ids), np.flatnonzero(keys >= 0))
