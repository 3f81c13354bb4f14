"""Batched registration (vicp_batch_*) against the oracle, pair by pair: every
pair's grid bit-exact (keys, offsets, CSR segments as sets, occupancy, root,
ring), every source point's neighbour as in the single-pair tests, and every
pair's registered pose within 1e-5 rad and 1e-5 x extent of the oracle's with
the same iteration count.  Also: the batched result equals the single-pair
path's at the same tolerance, runs are bit-identical (graph replay or direct
launches), every iteration kernel shape gives the same neighbours, the
autotuner, the host-input entry point, a degenerate pair among good ones, and
the full 256-pair workload (4.6M points) with the oracle on sampled pairs."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import assert_grid_equal, context, rot_err, to_np, vicp
from paper_2512_04996_gb300 import synth

pytestmark = pytest.mark.gpu

L = 10
ROT_TOL = 1e-5


def _pool(ps):
    tgt = np.ascontiguousarray(np.concatenate([p.target for p in ps]))
    src = np.ascontiguousarray(np.concatenate([p.source for p in ps]))
    n_tgt = np.array([p.target.shape[0] for p in ps], np.int32)
    n_src = np.array([p.source.shape[0] for p in ps], np.int32)
    vs = np.array([p.voxel_size for p in ps], np.float32)
    dv = np.array([p.grid_divisions for p in ps], np.int32)
    return tgt, src, n_tgt, n_src, vs, dv


def _batch(ps, **params):
    v = vicp()
    kw = dict(dilation_layers=L)
    kw.update(params)
    b = v.Batch(**kw)
    tgt, src, n_tgt, n_src, vs, dv = _pool(ps)
    t = torch.from_numpy(tgt).cuda()
    s = torch.from_numpy(src).cuda()
    b.build(t, n_tgt, vs, dv)
    return b, t, s, n_src


def _small(n_pairs=8, n_min=600, n_max=5000, seed=41):
    return synth.batched_pairs(seed=seed, n_pairs=n_pairs, n_min=n_min, n_max=n_max)


def _extent(target):
    t = target[:, :3]
    return float((t.max(0) - t.min(0)).max())


def _assert_pose_close(T, R, extent, tol=ROT_TOL):
    assert rot_err(T, R) <= tol, rot_err(T, R)
    assert np.linalg.norm(T[:3, 3] - R[:3, 3]) <= tol * extent


def _pair_grid_np(b, k):
    g = {key: to_np(val) for key, val in b.pair_grid(k).items()}
    g["offsets"] = (g["offsets"].astype(np.int64) - g["base"]).astype(np.uint32)
    return g


def test_batch_grids_equal_oracle():
    ps = _small(n_pairs=9, n_min=300, n_max=7000)
    b, *_ = _batch(ps)
    for k, p in enumerate(ps):
        g = _pair_grid_np(b, k)
        og = oracle.fit_grid(p.target, p.voxel_size, p.grid_divisions)
        assert g["origin"] == og.origin and g["voxel_size"] == og.h
        assert g["inv_voxel_size"] == og.inv_h and g["dims"] == og.dims
        ref = oracle.build_grid(og, p.target, L)
        assert_grid_equal(g, ref, p.target)


def test_batch_grids_single_point_and_coincident_targets():
    """Degenerate targets among ordinary ones: one point; all points in one
    voxel (a one-voxel grid)."""
    ps = _small(n_pairs=3, n_min=500, n_max=2000, seed=7)
    one = synth.Pair("one", ps[0].target[:1].copy(), ps[0].source[:50].copy(), np.eye(4), grid_divisions=64)
    same = np.tile(np.array([[0.2, -0.1, 0.4, 0.0]], np.float32), (300, 1))
    coin = synth.Pair("coincident", same, ps[1].source[:64].copy(), np.eye(4), grid_divisions=64)
    ps = [ps[0], one, ps[1], coin, ps[2]]
    b, *_ = _batch(ps)
    for k, p in enumerate(ps):
        g = _pair_grid_np(b, k)
        og = oracle.fit_grid(p.target, p.voxel_size, p.grid_divisions)
        assert g["dims"] == og.dims
        assert_grid_equal(g, oracle.build_grid(og, p.target, L), p.target)


@pytest.mark.parametrize("which", ["identity", "ground_truth"])
def test_batch_correspond_equals_oracle(which):
    from test_gpu_nns import _assert_nn_equal
    ps = _small(n_pairs=8, n_min=400, n_max=6000, seed=3)
    b, t, s, n_src = _batch(ps)
    T = np.stack([np.eye(4) if which == "identity" else p.T_gt for p in ps])
    nn, d2 = b.correspond(s, n_src, torch.from_numpy(np.ascontiguousarray(T)).cuda())
    nn, d2 = to_np(nn), to_np(d2)
    at = 0
    n_fb = 0
    for k, p in enumerate(ps):
        m = p.source.shape[0]
        og = oracle.fit_grid(p.target, p.voxel_size, p.grid_divisions)
        ref = oracle.build_grid(og, p.target, L)
        rnn, rd2, rfb = oracle.correspond(og, ref, p.target, p.source, T[k])
        _assert_nn_equal(nn[at:at + m], d2[at:at + m], rnn, rd2, p.target)
        n_fb += int(rfb.sum())
        at += m
    assert b.report(reset=True)["fallbacks"] == n_fb


@pytest.mark.parametrize("shape", range(7))
def test_every_shape_gives_the_same_neighbours(shape):
    ps = _small(n_pairs=6, n_min=900, n_max=9000, seed=11)
    T = torch.from_numpy(np.ascontiguousarray(np.stack([np.eye(4)] * len(ps)))).cuda()
    b0, t0, s0, n_src = _batch(ps, shape=0)
    nn0, d20 = b0.correspond(s0, n_src, T)
    b, t, s, _ = _batch(ps, shape=shape)
    nn, d2 = b.correspond(s, n_src, T)
    assert torch.equal(nn, nn0) and torch.equal(d2, d20)


def _prec_flags(prec):
    return vicp().VICP_BATCH_FLAG_FP64 if prec == "fp64" else 0


@pytest.mark.parametrize("prec", ["double_float", "fp64"])
def test_batch_register_matches_oracle(prec):
    ps = _small(n_pairs=6, n_min=500, n_max=4000, seed=19)
    iters = 12
    b, t, s, n_src = _batch(ps, max_iters=iters, rmse_eps=0.0, flags=_prec_flags(prec))
    st, T, it, rm, ps_status = b.register(s, n_src)
    assert st == 0 and (ps_status == 0).all() and (it == iters).all()
    for k, p in enumerate(ps):
        og = oracle.fit_grid(p.target, p.voxel_size, p.grid_divisions)
        rst, R, rit, hist = oracle.register(og, L, p.target, p.source, np.eye(4), max_iters=iters, eps=0.0)
        assert rst == 0 and rit == iters
        _assert_pose_close(T[k], R, _extent(p.target))
        assert abs(rm[k] - hist[-1]) <= 1e-7 * hist[-1]


def test_batch_stopping_rule_per_pair():
    """Each pair stops on its own |rmse_k - rmse_(k-1)| < eps (the paper's
    rule), at the oracle's iteration count."""
    ps = _small(n_pairs=5, n_min=800, n_max=3000, seed=23)
    b, t, s, n_src = _batch(ps, max_iters=50, rmse_eps=1e-5)
    st, T, it, rm, _ = b.register(s, n_src)
    assert st == 0
    for k, p in enumerate(ps):
        og = oracle.fit_grid(p.target, p.voxel_size, p.grid_divisions)
        rst, R, rit, hist = oracle.register(og, L, p.target, p.source, np.eye(4), max_iters=50, eps=1e-5)
        assert it[k] == rit and 2 <= rit < 50
        _assert_pose_close(T[k], R, _extent(p.target))


def test_batch_equals_single_pair_path():
    """Equal pose accuracy: each pair's batched pose against vicp_register on
    the pair alone."""
    ps = _small(n_pairs=6, n_min=1000, n_max=8000, seed=29)
    iters = 20
    b, t, s, n_src = _batch(ps, max_iters=iters)
    st, T, it, rm, _ = b.register(s, n_src)
    assert st == 0
    for k, p in enumerate(ps):
        ctx = context(L=L, voxel_size=p.voxel_size, divisions=p.grid_divisions, max_iters=iters, eps=0.0)
        sst, S, sit, srm = ctx.register(torch.from_numpy(p.source).cuda(), torch.from_numpy(p.target).cuda())
        assert sst == 0 and sit == it[k]
        _assert_pose_close(T[k], S, _extent(p.target))


@pytest.mark.parametrize("prec", ["double_float", "fp64"])
def test_batch_deterministic_graph_and_direct(prec):
    v = vicp()
    ps = _small(n_pairs=5, n_min=1000, n_max=6000, seed=31)
    b, t, s, n_src = _batch(ps, max_iters=8, flags=_prec_flags(prec))
    r1 = b.register(s, n_src)
    r2 = b.register(s, n_src)   # replayed graph
    bd, td, sd, _ = _batch(ps, max_iters=8, flags=v.VICP_BATCH_FLAG_NO_GRAPH | _prec_flags(prec))
    r3 = bd.register(sd, n_src)
    for r in (r2, r3):
        assert r[0] == 0 and np.array_equal(r[1], r1[1]) and np.array_equal(r[2], r1[2])
        assert np.array_equal(r[3], r1[3])
    assert b.launch_count() >= 2 * 8


def test_batch_initial_poses_and_host_entry():
    ps = _small(n_pairs=4, n_min=700, n_max=3000, seed=37)
    rng = np.random.default_rng(5)
    T0 = np.stack([synth.random_rigid(rng, 3.0, 0.02) for _ in ps])
    b, t, s, n_src = _batch(ps, max_iters=6)
    st, T, it, rm, _ = b.register(s, n_src, T0)
    tgt, src, n_tgt, n_src2, vs, dv = _pool(ps)
    bh = vicp().Batch(dilation_layers=L, max_iters=6)
    sth, Th, ith, rmh, _ = bh.register_host(src, n_src2, tgt, n_tgt, vs, dv, T0)
    assert st == 0 and sth == 0
    assert np.array_equal(T, Th) and np.array_equal(it, ith)
    for k, p in enumerate(ps):
        og = oracle.fit_grid(p.target, p.voxel_size, p.grid_divisions)
        rst, R, rit, _ = oracle.register(og, L, p.target, p.source, T0[k], max_iters=6, eps=0.0)
        _assert_pose_close(T[k], R, _extent(p.target))


def test_degenerate_pair_does_not_disturb_the_others():
    """A pair whose only source point makes rank(H) < 2 keeps its pose and
    reports VICP_ERR_DEGENERATE; its neighbours register normally."""
    v = vicp()
    ps = _small(n_pairs=3, n_min=800, n_max=2000, seed=43)
    lone = synth.Pair("lone", ps[1].target.copy(), ps[1].source[:1].copy(), np.eye(4), grid_divisions=64)
    ps = [ps[0], lone, ps[2]]
    b, t, s, n_src = _batch(ps, max_iters=5)
    st, T, it, rm, pst = b.register(s, n_src)
    assert st == 0
    assert pst[1] == v.VICP_ERR_DEGENERATE and np.array_equal(T[1], np.eye(4)) and it[1] == 0
    assert pst[0] == 0 and pst[2] == 0
    for k in (0, 2):
        p = ps[k]
        og = oracle.fit_grid(p.target, p.voxel_size, p.grid_divisions)
        rst, R, rit, _ = oracle.register(og, L, p.target, p.source, np.eye(4), max_iters=5, eps=0.0)
        _assert_pose_close(T[k], R, _extent(p.target))
    # without a per-pair status array the call itself reports it
    T0 = np.ascontiguousarray(np.tile(np.eye(4), (3, 1, 1)))
    import ctypes as C
    st2 = b._lib.vicp_batch_register(b.handle, s.data_ptr(), n_src.ctypes.data_as(C.c_void_p),
                                     T0.ctypes.data_as(C.c_void_p), None, None, None)
    assert st2 == v.VICP_ERR_DEGENERATE


def test_autotuner_picks_a_runnable_shape():
    v = vicp()
    ps = _small(n_pairs=6, n_min=2000, n_max=20000, seed=47)
    b, t, s, n_src = _batch(ps, max_iters=10)
    shape, ms = b.tune(s, n_src, iters=3, trials=2)
    assert 0 <= shape < v.VICP_BATCH_SHAPES
    assert ms[shape] > 0 and all(ms[shape] <= m for m in ms if m > 0)
    st, T, it, rm, _ = b.register(s, n_src)   # uses the tuned shape
    assert st == 0 and (it == 10).all()


def test_argument_checks():
    v = vicp()
    ps = _small(n_pairs=2, n_min=500, n_max=900, seed=53)
    tgt, src, n_tgt, n_src, vs, dv = _pool(ps)
    b = v.Batch(dilation_layers=L)
    s = torch.from_numpy(src).cuda()
    st = b.register(s, n_src)[0]
    assert st == v.VICP_ERR_STATE
    t = torch.from_numpy(tgt).cuda()
    with pytest.raises(v.VicpError) as e:
        b.build(t, np.array([n_tgt[0] + n_tgt[1], 0], np.int32), vs, dv)
    assert e.value.status == v.VICP_ERR_INVALID
    with pytest.raises(v.VicpError) as e:
        b.build(t, n_tgt, np.zeros(2, np.float32), np.zeros(2, np.int32))
    assert e.value.status == v.VICP_ERR_INVALID
    b.build(t, n_tgt, vs, dv)
    st = b.register(s, n_src)[0]
    assert st == 0


_FULL_ORACLE = {}


@pytest.mark.parametrize("prec", ["double_float", "fp64"])
def test_full_batched_workload_sampled(oracle_threads, prec):
    """The 256-pair workload (sizes log-uniform in 2k..64k, 4.6M points in
    all, 40 iterations) in the launch configuration of the benchmark; the
    oracle registers every sixteenth pair by size (from the smallest to the
    largest), and the single-pair GPU path every fourth pair."""
    ps = synth.batched_pairs()
    assert len(ps) == 256
    b, t, s, n_src = _batch(ps, max_iters=40, flags=_prec_flags(prec))
    st, T, it, rm, pst = b.register(s, n_src)
    assert st == 0 and (pst == 0).all() and (it == 40).all()
    sizes = np.array([p.source.shape[0] for p in ps])
    order = np.argsort(sizes)
    for k in [int(x) for x in order[::16]] + [int(order[-1])]:
        p = ps[k]
        if k not in _FULL_ORACLE:
            og = oracle.fit_grid(p.target, p.voxel_size, p.grid_divisions)
            _FULL_ORACLE[k] = oracle.register(og, L, p.target, p.source, np.eye(4), max_iters=40, eps=0.0)
        rst, R, rit, hist = _FULL_ORACLE[k]
        _assert_pose_close(T[k], R, _extent(p.target))
    single_flags = vicp().VICP_FLAG_FP64_SOLVE if prec == "fp64" else 0
    for k in range(0, 256, 4):
        p = ps[k]
        ctx = context(L=L, voxel_size=p.voxel_size, divisions=p.grid_divisions, max_iters=40, eps=0.0,
                      flags=single_flags)
        sst, S, sit, _ = ctx.register(torch.from_numpy(p.source).cuda(), torch.from_numpy(p.target).cuda())
        assert sst == 0
        _assert_pose_close(T[k], S, _extent(p.target))


def test_more_pairs_than_the_shared_memory_tables_hold():
    """2,100 small pairs (the dilation's per-pair unit tables then stay in
    global memory): sampled pairs' grids and registrations against the
    oracle."""
    rng = np.random.default_rng(79)
    ps = [synth.sphere_plane(seed=int(rng.integers(0, 2**31 - 1)), n=int(rng.integers(120, 400)), max_deg=10.0,
                             max_trans=0.05) for _ in range(2100)]
    iters = 4
    b, t, s, n_src = _batch(ps, max_iters=iters)
    st, T, it, rm, pst = b.register(s, n_src)
    assert st == 0 and (it == iters).all()
    for k in (0, 1, 1023, 2047, 2048, 2099):
        p = ps[k]
        g = _pair_grid_np(b, k)
        og = oracle.fit_grid(p.target, p.voxel_size, p.grid_divisions)
        assert_grid_equal(g, oracle.build_grid(og, p.target, L), p.target)
        _, R, _, _ = oracle.register(og, L, p.target, p.source, np.eye(4), max_iters=iters, eps=0.0)
        _assert_pose_close(T[k], R, _extent(p.target))


def test_rebuild_reads_only_the_offsets_it_writes():
    """As the single-grid test: a batch built and viewed (completed offsets)
    on one set of targets, rebuilt on other targets with the same pair sizes
    and searched without a view in between, finds the oracle's neighbours."""
    from test_gpu_nns import _assert_nn_equal
    ps = _small(n_pairs=6, n_min=500, n_max=5000, seed=19)
    b, t, s, n_src = _batch(ps)
    dims = [b.pair_grid(k)["dims"] for k in range(len(ps))]
    ps2 = []
    for p in ps:   # each target mirrored in x and y inside its own box: other voxels, same grid
        tgt = p.target.copy()
        lo, hi = tgt[:, :2].min(0), tgt[:, :2].max(0)
        tgt[:, :2] = (lo + hi) - tgt[:, :2]
        ps2.append(synth.Pair(p.name, tgt, p.source, p.T_gt, voxel_size=p.voxel_size,
                              grid_divisions=p.grid_divisions))
    b2, *_ = _batch(ps2)
    assert [b2.pair_grid(k)["dims"] for k in range(len(ps))] == dims   # b's pooled arrays will be reused
    tgt2, _, n_tgt, _, vs, dv = _pool(ps2)
    b.build(torch.from_numpy(tgt2).cuda(), n_tgt, vs, dv)
    T = np.stack([p.T_gt for p in ps2])
    nn, d2 = b.correspond(s, n_src, torch.from_numpy(np.ascontiguousarray(T)).cuda())
    nn, d2 = to_np(nn), to_np(d2)
    at = 0
    for k, p in enumerate(ps2):
        m = p.source.shape[0]
        og = oracle.fit_grid(p.target, p.voxel_size, p.grid_divisions)
        ref = oracle.build_grid(og, p.target, L)
        rnn, rd2, _ = oracle.correspond(og, ref, p.target, p.source, T[k])
        _assert_nn_equal(nn[at:at + m], d2[at:at + m], rnn, rd2, p.target)
        at += m
    g = _pair_grid_np(b, 2)
    og = oracle.fit_grid(ps2[2].target, ps2[2].voxel_size, ps2[2].grid_divisions)
    assert np.array_equal(g["offsets"], oracle.build_grid(og, ps2[2].target, L)["off"])
