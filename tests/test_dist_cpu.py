"""The benchmark's multi-process path on CPU: two gloo ranks initialise from
the torchrun environment variables, meet at the barrier and agree on the
slowest rank's time (the path runs independent replicas, so this is the only
communication)."""
import os
import socket

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
