"""The benchmark's multi-process paths on CPU.  Two gloo ranks initialise from
the torchrun environment variables, meet at the barrier and agree on the
slowest rank's time (the scene workload runs independent replicas, so this is
its only communication); and batched registration sharded by pair: every pair
goes to exactly one rank, the ranks' shares are balanced, and the poses
gathered from two ranks equal the single-rank result."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    torch.cuda.is_available = lambda: False   # gloo ranks on CPU, also on a GPU machine
    import bench
    r, ws, local = bench._dist_init()
    assert (r, ws, local) == (rank, world, rank)
    bench._barrier(ws)
    t = bench._max_over_ranks(1.5 + rank, ws)
    out.put((rank, t))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_ranks_agree_on_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got == {0: 2.5, 1: 2.5}


def test_single_process_needs_no_group():
    import bench
    os.environ.pop("WORLD_SIZE", None)
    assert bench._dist_init() == (0, 1, 0)
    assert bench._max_over_ranks(3.25, 1) == 3.25


# ---------------------------------------------------------------------------
# batched registration sharded by pair: partition and gather on two gloo ranks
# ---------------------------------------------------------------------------
def test_partition_covers_every_pair_once_and_balances():
    from paper_2512_04996_gb300 import shard
    # sizes like the batched workload's: log-uniform in 2k..64k points per side
    work = [2 * int(x) for x in np.exp(np.random.default_rng(4).uniform(np.log(2000), np.log(64000), 256))]
    for ws in (1, 2, 3, 8):
        parts = shard.partition_pairs(work, ws)
        flat = sorted(k for part in parts for k in part)
        assert flat == list(range(256))
        loads = [sum(work[k] for k in part) for part in parts]
        # greedy largest-first: no rank exceeds the mean by more than the largest pair
        assert max(loads) <= sum(work) / ws + max(work)
        assert parts == shard.partition_pairs(work, ws)   # deterministic


def _fake_register(pairs):
    """A stand-in for one rank's batched registration: a pose that encodes the
    pair index (the gather must put it back in its place)."""
    poses = np.stack([np.eye(4) + 1e-3 * k for k in pairs]) if pairs else np.zeros((0, 4, 4))
    return poses, np.array([10 + k % 7 for k in pairs], np.int32)


def _shard_rank(rank, world, port, work, out):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    torch.cuda.is_available = lambda: False
    import bench
    from paper_2512_04996_gb300 import shard
    r, ws, _ = bench._dist_init()
    mine = shard.partition_pairs(work, ws)[r]
    P, it = _fake_register(mine)
    poses, iters = shard.gather_results(mine, P, it, len(work), ws)
    out.put((r, len(mine), poses, iters))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_ranks_gather_the_single_rank_result():
    from paper_2512_04996_gb300 import shard
    work = list(np.random.default_rng(3).integers(2000, 64000, 37))
    ref_poses, ref_iters = shard.gather_results(list(range(37)), *_fake_register(list(range(37))), 37, 1)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, work, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert sum(n for _, n, _, _ in got) == 37 and all(n > 0 for _, n, _, _ in got)
    for _, _, poses, iters in got:
        assert np.array_equal(poses, ref_poses) and np.array_equal(iters, ref_iters)


def test_gather_rejects_a_missing_pair():
    from paper_2512_04996_gb300 import shard
    with pytest.raises(RuntimeError):
        shard.gather_results([0, 2], np.zeros((2, 4, 4)), [1, 1], 3, 1)
