"""GPU ICP iterations (vicp_step / vicp_register) against the oracle: the pose
within 1e-5 rad and 1e-5 x extent, the same iteration count under the
paper's stopping rule, deterministic results, and the degenerate case."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import context, gpu_grid, oracle_grid_for, rot_err, to_np
from paper_2512_04996_gb300.synth import random_rigid

pytestmark = pytest.mark.gpu

ROT_TOL = 1e-5
PRECISIONS = ["double_float", "fp64"]


def _prec_flags(prec):
    from paper_2512_04996_gb300 import vicp
    return vicp.VICP_FLAG_FP64_SOLVE if prec == "fp64" else 0


def _extent(target):
    t = target[:, :3]
    return float((t.max(0) - t.min(0)).max())


def _assert_pose_close(T, R, extent):
    assert rot_err(T, R) <= ROT_TOL, rot_err(T, R)
    assert np.linalg.norm(T[:3, 3] - R[:3, 3]) <= 1e-5 * extent


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("k", [1, 2, 3])
def test_single_step(pairs, k, prec):
    """One step at a pose: the same correspondences as the oracle, so the
    update differs only by the rounding of the sums and the solve -- within
    the pose tolerance for double-float, and within 1e-9 rad / 1e-9 x extent
    and 1e-12 relative RMSE for FP64."""
    p = pairs(k)
    ctx, g = gpu_grid(p.target, L=10, voxel_size=p.voxel_size, divisions=p.grid_divisions,
                      flags=_prec_flags(prec))
    grid, ref = oracle_grid_for(g, p.target, 10)
    T0 = np.eye(4) if k != 1 else random_rigid(np.random.default_rng(9), 3.0, 0.02)
    pose = torch.from_numpy(T0.copy()).cuda()
    rmse = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.step(torch.from_numpy(p.source).cuda(), pose, rmse)
    assert ctx.sync() == 0
    st, R, r_rmse, *_ = oracle.iterate(grid, ref, p.target, p.source, T0)
    assert st == 0
    T = to_np(pose)
    _assert_pose_close(T, R, _extent(p.target))
    if prec == "fp64":
        assert rot_err(T, R) <= 1e-9 and np.linalg.norm(T[:3, 3] - R[:3, 3]) <= 1e-9 * _extent(p.target)
        assert abs(float(to_np(rmse)[0]) - r_rmse) <= 1e-12 * r_rmse
    else:
        assert abs(float(to_np(rmse)[0]) - r_rmse) <= 1e-9 * r_rmse


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("k", [1, 2])
def test_register_fixed_iterations(pairs, k, prec):
    p = pairs(k)
    ctx = context(L=10, voxel_size=p.voxel_size, divisions=p.grid_divisions, max_iters=p.iters, eps=0.0,
                  flags=_prec_flags(prec))
    st, T, it, rm = ctx.register(torch.from_numpy(p.source).cuda(), torch.from_numpy(p.target).cuda())
    assert st == 0 and it == p.iters
    grid = oracle.fit_grid(p.target, p.voxel_size, p.grid_divisions)
    rst, R, rit, hist = oracle.register(grid, 10, p.target, p.source, np.eye(4), max_iters=p.iters, eps=0.0)
    assert rst == 0 and rit == it
    _assert_pose_close(T, R, _extent(p.target))
    assert abs(rm - hist[-1]) <= 1e-7 * hist[-1]


_SCENE_ORACLE = {}


def _scene_oracle(p, max_iters, eps):
    key = (max_iters, eps)
    if key not in _SCENE_ORACLE:
        grid = oracle.fit_grid(p.target, p.voxel_size, 0)
        _SCENE_ORACLE[key] = oracle.register(grid, 10, p.target, p.source, np.eye(4), max_iters=max_iters, eps=eps)
    return _SCENE_ORACLE[key]


@pytest.mark.parametrize("prec", PRECISIONS)
def test_register_scene_thirty_iterations_rebuilding_each(pairs, oracle_threads, prec):
    """The benchmark's configuration end to end: the 226k-point scene, grid
    rebuilt and dilated every iteration, 30 iterations from the identity,
    against the oracle's 30 iterations (pose, iteration count, RMSE)."""
    from paper_2512_04996_gb300 import vicp
    p = pairs(3)
    ctx = context(L=10, voxel_size=p.voxel_size, max_iters=30, eps=0.0,
                  flags=vicp.VICP_FLAG_KEEP_GRID | vicp.VICP_FLAG_REBUILD_EACH_ITER | _prec_flags(prec))
    st, T, it, rm = ctx.register(torch.from_numpy(p.source).cuda(), torch.from_numpy(p.target).cuda())
    assert st == 0 and it == 30
    rst, R, rit, hist = _scene_oracle(p, 30, 0.0)
    assert rst == 0 and rit == it
    _assert_pose_close(T, R, _extent(p.target))
    assert abs(rm - hist[-1]) <= 1e-7 * hist[-1]


@pytest.mark.parametrize("prec", PRECISIONS)
def test_register_scene_paper_stopping_rule(pairs, oracle_threads, prec):
    """The scene under the paper's stopping rule (RMSE difference 1e-5, at
    most 50 iterations): the same iteration count and pose as the oracle."""
    p = pairs(3)
    ctx = context(L=10, voxel_size=p.voxel_size, max_iters=50, eps=1e-5, flags=_prec_flags(prec))
    st, T, it, rm = ctx.register(torch.from_numpy(p.source).cuda(), torch.from_numpy(p.target).cuda())
    rst, R, rit, hist = _scene_oracle(p, 50, 1e-5)
    assert st == 0 and rst == 0 and it == rit and 2 <= it <= 50
    _assert_pose_close(T, R, _extent(p.target))
    assert abs(rm - hist[-1]) <= 1e-7 * hist[-1]


def test_paper_stopping_rule(pairs):
    from paper_2512_04996_gb300 import synth
    p = synth.sphere_plane(seed=77, n=2000)
    ctx = context(L=10, divisions=64, max_iters=50, eps=1e-5)
    st, T, it, rm = ctx.register(torch.from_numpy(p.source).cuda(), torch.from_numpy(p.target).cuda())
    grid = oracle.fit_grid(p.target, 0.0, 64)
    rst, R, rit, hist = oracle.register(grid, 10, p.target, p.source, np.eye(4), max_iters=50, eps=1e-5)
    assert st == 0 and it == rit and 2 <= it < 50
    _assert_pose_close(T, R, _extent(p.target))


def test_deterministic(pairs):
    p = pairs(2)
    out = []
    for _ in range(2):
        ctx = context(L=10, divisions=128, max_iters=8, eps=0.0)
        out.append(ctx.register(torch.from_numpy(p.source).cuda(), torch.from_numpy(p.target).cuda()))
    assert out[0][0] == out[1][0] == 0
    assert np.array_equal(out[0][1], out[1][1]) and out[0][3] == out[1][3]


def test_register_host_equals_register(pairs):
    p = pairs(1)
    ctx = context(L=10, divisions=64, max_iters=10, eps=0.0)
    a = ctx.register(torch.from_numpy(p.source).cuda(), torch.from_numpy(p.target).cuda())
    b = ctx.register_host(p.source, p.target)
    assert a[0] == b[0] == 0 and a[2] == b[2]
    assert np.array_equal(a[1], b[1])


def test_rebuild_each_iteration_equals_build_once(pairs):
    from paper_2512_04996_gb300 import vicp
    p = pairs(1)
    res = []
    for flags in (0, vicp.VICP_FLAG_KEEP_GRID | vicp.VICP_FLAG_REBUILD_EACH_ITER):
        ctx = context(L=10, divisions=64, max_iters=12, eps=0.0, flags=flags)
        res.append(ctx.register(torch.from_numpy(p.source).cuda(), torch.from_numpy(p.target).cuda()))
    assert np.array_equal(res[0][1], res[1][1])


def test_steps_equal_register(pairs):
    p = pairs(1)
    ctx = context(L=10, divisions=64, max_iters=5, eps=0.0)
    st, T, it, rm = ctx.register(torch.from_numpy(p.source).cuda(), torch.from_numpy(p.target).cuda())
    ctx2, g = gpu_grid(p.target, L=10, divisions=64)
    pose = torch.eye(4, dtype=torch.float64, device="cuda").contiguous()
    src = torch.from_numpy(p.source).cuda()
    for _ in range(5):
        ctx2.step(src, pose)
    assert ctx2.sync() == 0
    assert np.array_equal(to_np(pose), T)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_degenerate_geometry_reports_and_keeps_pose(prec):
    from paper_2512_04996_gb300 import vicp
    tgt = np.zeros((500, 4), np.float32)
    tgt[:, 0] = np.linspace(0, 1, 500)
    ctx = context(L=4, divisions=16, max_iters=5, eps=0.0, flags=_prec_flags(prec))
    st, T, it, rm = ctx.register(torch.from_numpy(tgt).cuda(), torch.from_numpy(tgt).cuda())
    assert st == vicp.VICP_ERR_DEGENERATE and it == 0
    assert np.array_equal(T, np.eye(4))
    grid = oracle.fit_grid(tgt, 0.0, 16)
    rst, R, rit, hist = oracle.register(grid, 4, tgt, tgt, np.eye(4), max_iters=5, eps=0.0)
    assert rst == oracle.ERR_DEGENERATE and rit == 0
    # the context stays usable
    p = np.zeros((300, 4), np.float32)
    p[:, :3] = np.random.default_rng(0).standard_normal((300, 3))
    st, T, it, rm = ctx.register(torch.from_numpy(p).cuda(), torch.from_numpy(p).cuda())
    assert st == 0 and np.abs(T - np.eye(4)).max() < 1e-12


def test_profile_counts_launches(pairs):
    p = pairs(1)
    ctx, g = gpu_grid(p.target, L=10, divisions=64)
    ctx.profile_enable(True)
    pose = torch.eye(4, dtype=torch.float64, device="cuda").contiguous()
    src = torch.from_numpy(p.source).cuda()
    before = ctx.launch_count()
    for _ in range(3):
        ctx.step(src, pose)
    prof = ctx.profile_read()
    assert ctx.launch_count() - before == 9
    for name in ("correspond", "fallback", "reduce_solve"):
        assert prof[name][0] == 3 and prof[name][1] > 0.0


def test_fp64_and_double_float_agree_and_are_deterministic(pairs):
    """The two precisions register the object workload to the same pose
    (both within the oracle's tolerance of each other), and each gives
    bit-identical results from run to run."""
    p = pairs(2)
    out = {}
    for prec in ("double_float", "double_float", "fp64", "fp64"):
        ctx = context(L=10, divisions=128, max_iters=10, eps=0.0, flags=_prec_flags(prec))
        st, T, it, rm = ctx.register(torch.from_numpy(p.source).cuda(), torch.from_numpy(p.target).cuda())
        assert st == 0 and it == 10
        if prec in out:
            assert np.array_equal(out[prec][0], T) and out[prec][1] == rm
        out[prec] = (T, rm)
    _assert_pose_close(out["fp64"][0], out["double_float"][0], _extent(p.target))


def _graph_pair(p, flags, max_iters, voxel_size=None):
    from paper_2512_04996_gb300 import vicp
    kw = dict(L=10, voxel_size=p.voxel_size if voxel_size is None else voxel_size, divisions=p.grid_divisions,
              max_iters=max_iters, eps=0.0)
    return (context(flags=flags, **kw), context(flags=flags | vicp.VICP_FLAG_NO_GRAPH, **kw))


@pytest.mark.parametrize("k,max_iters,rebuild", [(1, 30, False), (1, 3, True), (2, 1, True), (3, 2, True)])
def test_register_graph_replays_equal_direct_launches(pairs, k, max_iters, rebuild):
    """vicp_register replayed from its captured graph (from the second call
    with the same arguments on) gives the direct launches' results bit for
    bit, whatever the initial pose, with an odd or even number of builds per
    call (the double-buffered build state)."""
    from paper_2512_04996_gb300 import vicp
    p = pairs(k)
    flags = vicp.VICP_FLAG_KEEP_GRID | (vicp.VICP_FLAG_REBUILD_EACH_ITER if rebuild else 0)
    g, d = _graph_pair(p, flags, max_iters)
    src, tgt = torch.from_numpy(p.source).cuda(), torch.from_numpy(p.target).cuda()
    rng = np.random.default_rng(20 + k)
    for call in range(4):
        T0 = random_rigid(rng, 4.0, 0.02) if call % 2 else np.eye(4)
        a, b = g.register(src, tgt, T0), d.register(src, tgt, T0)
        assert a[0] == b[0] == 0 and a[2] == b[2] and a[3] == b[3], call
        assert np.array_equal(a[1], b[1]), call
        assert g.graph_replayed() == (call >= 1) and not d.graph_replayed(), call
    # a grid view after the replays is the direct context's
    ga, gb = g.get_grid(), d.get_grid()
    for key in ("keys", "offsets", "root", "ring", "occupancy"):
        assert torch.equal(ga[key], gb[key]), key


def test_register_host_graph_reads_the_clouds_anew(pairs):
    """vicp_register_host replayed from a graph copies the host clouds at
    every replay: new contents at the same (page-locked) addresses give the
    results of direct launches on the new contents."""
    from paper_2512_04996_gb300 import vicp
    p = pairs(2)
    flags = vicp.VICP_FLAG_KEEP_GRID
    g, d = _graph_pair(p, flags, 5)
    src = torch.from_numpy(p.source.copy()).pin_memory()
    tgt = torch.from_numpy(p.target.copy()).pin_memory()
    s_np, t_np = src.numpy(), tgt.numpy()
    rng = np.random.default_rng(5)
    for call in range(4):
        if call == 3:   # move the source cloud in place
            s_np[:, :3] += np.float32(0.01)
        a, b = g.register_host(s_np, t_np), d.register_host(s_np, t_np)
        assert a[0] == b[0] == 0 and a[2] == b[2] and np.array_equal(a[1], b[1]), call
    # and the last result is the oracle's on the moved cloud
    grid = oracle.fit_grid(p.target, p.voxel_size, p.grid_divisions)
    rst, R, rit, hist = oracle.register(grid, 10, t_np, s_np, np.eye(4), max_iters=5, eps=0.0)
    _assert_pose_close(a[1], R, _extent(p.target))


def test_graph_and_direct_calls_interleave_on_one_context(pairs):
    """Captured and direct calls of every kind on one context: host
    registrations (captured from the second call, then replayed), then
    device-resident registrations, a plain search and host registrations
    again.  Each result equals that of a context that never captures."""
    from paper_2512_04996_gb300 import vicp
    p = pairs(2)
    g, d = _graph_pair(p, vicp.VICP_FLAG_KEEP_GRID, 3)
    s_np = torch.from_numpy(p.source.copy()).pin_memory().numpy()
    t_np = torch.from_numpy(p.target.copy()).pin_memory().numpy()
    src, tgt = torch.from_numpy(p.source).cuda(), torch.from_numpy(p.target).cuda()
    pose = torch.from_numpy(random_rigid(np.random.default_rng(3), 3.0, 0.02)).cuda()

    def both(call):
        a, b = call(g), call(d)
        assert a[0] == b[0] == 0 and a[2] == b[2] and np.array_equal(a[1], b[1])

    for _ in range(3):
        both(lambda c: c.register_host(s_np, t_np))
    for _ in range(3):
        both(lambda c: c.register(src, tgt))
    na, da, fa = g.correspond(src, pose)
    nb, db, fb = d.correspond(src, pose)
    assert torch.equal(na, nb) and torch.equal(da, db) and torch.equal(fa, fb)
    for _ in range(3):
        both(lambda c: c.register_host(s_np, t_np))
    for _ in range(2):
        both(lambda c: c.register(src, tgt))
