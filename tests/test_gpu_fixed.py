"""The fixed-capacity voxel store (vicp_fixed_build / vicp_fixed_correspond)
against the oracle and against the CSR store.

With a capacity of the largest voxel count nothing is dropped: every
neighbour equals the oracle's (equal index, or squared distance within 1e-6
relative) and the CSR path's bit for bit, on all three workloads.

With a smaller capacity the store keeps min(count, C) points of each voxel;
which ones depends on the order of the scatter's atomics, so the test reads
back the kept points, checks that they are a valid truncation (each lies in
its voxel, none twice, exactly min(count, C) per voxel, the dropped total
equals sum(max(0, count - C)) over the oracle's histogram), builds the
oracle's CSR of exactly those points and holds every neighbour to the
oracle's search over it (the root labels and the global search are the full
build's, as the store replaces only the voxel segments)."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import assert_nn_equal, gpu_grid, oracle_grid_for, to_np, vicp
from paper_2512_04996_gb300.synth import random_rigid

pytestmark = pytest.mark.gpu


def _searches(ctx, src, T):
    s = torch.from_numpy(np.ascontiguousarray(src)).cuda()
    pose = torch.from_numpy(np.ascontiguousarray(T, dtype=np.float64)).cuda()
    a = [to_np(x) for x in ctx.correspond(s, pose)]
    b = [to_np(x) for x in ctx.fixed_correspond(s, pose)]
    return a, b


@pytest.mark.parametrize("k", [1, 2, 3])
def test_capacity_of_the_largest_voxel_matches_oracle(pairs, oracle_threads, k):
    p = pairs(k)
    ctx, g = gpu_grid(p.target, L=10, voxel_size=p.voxel_size, divisions=p.grid_divisions)
    grid, ref = oracle_grid_for(g, p.target, 10)
    rep = ctx.memory_report()
    C = rep["max_voxel_count"]
    assert C == int(ref["counts"].max())
    over, nbytes = ctx.fixed_build(g["_target"], C)
    assert over == 0
    assert nbytes == g["n_voxels"] * C * 16 + 4 * g["n_voxels"]
    for T in (np.eye(4), p.T_gt, random_rigid(np.random.default_rng(k), 20.0, 0.2)):
        (nn, d2, nf), (fnn, fd2, fnf) = _searches(ctx, p.source, T)
        rnn, rd2, rfb = oracle.correspond(grid, ref, p.target, p.source, T)
        assert_nn_equal(fnn, fd2, rnn, rd2)
        assert int(fnf[0]) == int(rfb.sum())
        # and the CSR path's answers bit for bit
        assert np.array_equal(nn, fnn) and np.array_equal(d2.view(np.uint32), fd2.view(np.uint32))
        assert int(nf[0]) == int(fnf[0])


def _kept_csr(ctx, keys, counts, C):
    """The oracle-layout CSR (offsets, ids ascending per voxel) of the points
    the fixed store kept, after checking that they are a valid truncation."""
    fv = ctx.fixed_view()
    assert fv["capacity"] == C
    fill = to_np(fv["fill"]).astype(np.int64)
    assert np.array_equal(fill, counts.astype(np.int64))        # every point was counted in its voxel
    kept = np.minimum(fill, C)
    V = counts.shape[0]
    slot_ids = to_np(fv["slots"])[:, 3].view(np.int32).reshape(V, C)
    used = np.arange(C)[None, :] < kept[:, None]
    vox = np.repeat(np.arange(V), C).reshape(V, C)[used]
    ids = slot_ids[used]
    assert np.all((ids >= 0) & (ids < keys.shape[0]))
    assert np.array_equal(keys[ids], vox)                       # each kept point lies in its voxel
    assert np.unique(ids).shape[0] == ids.shape[0]              # none twice
    order = np.lexsort((ids, vox))                              # voxel order, ascending index inside
    off = np.zeros(V + 1, np.uint32)
    off[1:] = np.cumsum(kept).astype(np.uint32)
    return off, np.ascontiguousarray(ids[order].astype(np.int32))


@pytest.mark.parametrize("k", [1, 2])
def test_small_capacity_matches_oracle_on_kept_points(pairs, k):
    p = pairs(k)
    ctx, g = gpu_grid(p.target, L=10, voxel_size=p.voxel_size, divisions=p.grid_divisions)
    grid, ref = oracle_grid_for(g, p.target, 10)
    counts = ref["counts"]
    C = max(1, int(counts.max()) // 4)
    over, _ = ctx.fixed_build(g["_target"], C)
    assert over == int(np.maximum(counts.astype(np.int64) - C, 0).sum()) and over > 0
    off_t, ids_t = _kept_csr(ctx, ref["keys"], counts, C)
    trunc = dict(off=off_t, ids=ids_t, root=ref["root"])
    for T in (p.T_gt, random_rigid(np.random.default_rng(10 + k), 15.0, 0.1)):
        (nn, d2, nf), (fnn, fd2, fnf) = _searches(ctx, p.source, T)
        rnn, rd2, rfb = oracle.correspond(grid, trunc, p.target, p.source, T)
        assert_nn_equal(fnn, fd2, rnn, rd2)
        assert int(fnf[0]) == int(rfb.sum())
        # a truncated segment never gives a closer point than the full one
        assert np.all(fd2[~rfb] >= d2[~rfb])


def test_fixed_store_argument_checks(pairs):
    v = vicp()
    p = pairs(1)
    ctx = v.Context(v.default_params(grid_divisions=64))
    t = torch.from_numpy(p.target).cuda()
    with pytest.raises(v.VicpError) as e:
        ctx.fixed_build(t, 8)
    assert e.value.status == v.VICP_ERR_STATE
    with pytest.raises(v.VicpError) as e:
        ctx.fixed_view()
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
