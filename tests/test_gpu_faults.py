"""Failure handling without faulting the GPU: an allocator that returns NULL
gives VICP_ERR_OOM and leaks nothing; calls out of order return
VICP_ERR_STATE; an oversized grid is refused before any launch; the batched
iteration kernel's grid barrier (the library's only device-side wait) gives
up after its time limit with VICP_ERR_TIMEOUT when a block never arrives, and
the context works normally afterwards."""
import ctypes as C

import numpy as np
import pytest
import torch

from gpu_util import assert_grid_equal, context, gpu_grid, oracle_grid_for, to_np, vicp

pytestmark = pytest.mark.gpu


def test_allocator_failure_is_reported_and_nothing_leaks(pairs):
    v = vicp()
    live = {}
    budget = {"n": 6}

    @v.ALLOC_FN
    def alloc(nbytes, stream, user):
        if budget["n"] == 0:
            return None
        budget["n"] -= 1
        t = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        live[t.data_ptr()] = t
        return t.data_ptr()

    @v.FREE_FN
    def free(ptr, nbytes, stream, user):
        live.pop(ptr)

    a = v.vicp_allocator(alloc, free, None)
    ctx = v.Context(v.default_params(grid_divisions=64), allocator=a)
    with pytest.raises(v.VicpError) as e:
        ctx.build_grid(torch.from_numpy(pairs(1).target).cuda())
    assert e.value.status == v.VICP_ERR_OOM
    assert len(live) > 0
    ctx.close()
    assert live == {}


def test_torch_allocator_path_is_exact(pairs):
    """The same build with every workspace buffer from torch's allocator."""
    v = vicp()
    live = {}

    @v.ALLOC_FN
    def alloc(nbytes, stream, user):
        t = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        live[t.data_ptr()] = t
        return t.data_ptr()

    @v.FREE_FN
    def free(ptr, nbytes, stream, user):
        live.pop(ptr)

    p = pairs(1)
    a = v.vicp_allocator(alloc, free, None)
    ctx = v.Context(v.default_params(grid_divisions=64, dilation_layers=10), allocator=a)
    ctx.build_grid(torch.from_numpy(p.target).cuda())
    ctx.dilate(10)
    g = {k: to_np(x) for k, x in ctx.get_grid().items()}
    grid, ref = oracle_grid_for(g, p.target, 10)
    assert_grid_equal(g, ref, p.target)
    rep = ctx.memory_report()
    assert rep["current_bytes"] == sum(t.numel() for t in live.values())
    ctx.close()
    assert live == {}


def test_call_order_and_argument_errors(pairs):
    v = vicp()
    ctx = context(L=10, divisions=64)
    src = torch.from_numpy(pairs(1).source).cuda()
    pose = torch.eye(4, dtype=torch.float64, device="cuda").contiguous()
    with pytest.raises(v.VicpError) as e:
        ctx.step(src, pose)
    assert e.value.status == v.VICP_ERR_STATE
    with pytest.raises(v.VicpError) as e:
        ctx.dilate(5)
    assert e.value.status == v.VICP_ERR_STATE
    ctx.build_grid(torch.from_numpy(pairs(1).target).cuda())
    with pytest.raises(v.VicpError) as e:
        ctx.dilate(32)
    assert e.value.status == v.VICP_ERR_INVALID
    lib = v.load_library()
    misaligned = src.view(-1)[1:].data_ptr()
    assert lib.vicp_build_grid(ctx.handle, misaligned, 10) == v.VICP_ERR_INVALID
    assert lib.vicp_build_grid(ctx.handle, src.data_ptr(), 0) == v.VICP_ERR_INVALID
    assert ctx.sync() == 0


def test_grid_too_large_is_rejected():
    v = vicp()
    ctx = context(L=10, voxel_size=1.0, origin=(0, 0, 0), dims=(2048, 2048, 1024))
    with pytest.raises(v.VicpError) as e:
        ctx.build_grid(torch.zeros((4, 4), dtype=torch.float32, device="cuda"))
    assert e.value.status == v.VICP_ERR_GRID_TOO_LARGE


def test_batch_barrier_time_limit_and_recovery():
    """A test hook makes block 0 of the iteration kernel leave before the
    first grid barrier (nothing else ever arrives for it): the other blocks'
    wait runs out after one second, the call reports VICP_ERR_TIMEOUT, and
    the same context then registers exactly like a fresh one."""
    import time

    from paper_2512_04996_gb300 import synth
    v = vicp()
    ps = synth.batched_pairs(seed=61, n_pairs=3, n_min=800, n_max=2500)
    tgt = torch.from_numpy(np.concatenate([p.target for p in ps])).cuda()
    src = torch.from_numpy(np.concatenate([p.source for p in ps])).cuda()
    n_tgt = np.array([p.target.shape[0] for p in ps], np.int32)
    n_src = np.array([p.source.shape[0] for p in ps], np.int32)
    dv = np.array([p.grid_divisions for p in ps], np.int32)
    b = v.Batch(dilation_layers=10, max_iters=3, flags=v.VICP_BATCH_FLAG_TEST_BARRIER_TIMEOUT)
    b.build(tgt, n_tgt, None, dv)
    t0 = time.perf_counter()
    st = b.register(src, n_src)[0]
    assert st == v.VICP_ERR_TIMEOUT
    assert 0.9 < time.perf_counter() - t0 < 30.0
    b.set_flags(0)
    st, T, it, rm, _ = b.register(src, n_src)
    fresh = v.Batch(dilation_layers=10, max_iters=3)
    fresh.build(tgt, n_tgt, None, dv)
    st2, T2, it2, rm2, _ = fresh.register(src, n_src)
    assert st == 0 and st2 == 0
    assert np.array_equal(T, T2) and np.array_equal(it, it2) and np.array_equal(rm, rm2)


def test_batch_allocator_serves_every_buffer_and_failure_is_reported():
    """A batch context on a caller's allocator: registration works with every
    buffer from the allocator, destroy returns them all, and an allocator
    that runs dry gives VICP_ERR_OOM without leaking."""
    from paper_2512_04996_gb300 import synth
    v = vicp()
    live = {}
    budget = {"n": 10 ** 6}

    @v.ALLOC_FN
    def alloc(nbytes, stream, user):
        if budget["n"] == 0:
            return None
        budget["n"] -= 1
        t = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        live[t.data_ptr()] = t
        return t.data_ptr()

    @v.FREE_FN
    def free(ptr, nbytes, stream, user):
        live.pop(ptr)

    a = v.vicp_allocator(alloc, free, None)
    ps = synth.batched_pairs(seed=67, n_pairs=3, n_min=800, n_max=2500)
    tgt = torch.from_numpy(np.concatenate([p.target for p in ps])).cuda()
    src = torch.from_numpy(np.concatenate([p.source for p in ps])).cuda()
    n_tgt = np.array([p.target.shape[0] for p in ps], np.int32)
    n_src = np.array([p.source.shape[0] for p in ps], np.int32)
    dv = np.array([p.grid_divisions for p in ps], np.int32)
    b = v.Batch(v.batch_default_params(max_iters=3), allocator=a)
    b.build(tgt, n_tgt, None, dv)
    st = b.register(src, n_src)[0]
    assert st == 0 and len(live) > 10
    b.close()
    assert live == {}
    budget["n"] = 8
    b = v.Batch(v.batch_default_params(max_iters=3), allocator=a)
    with pytest.raises(v.VicpError) as e:
        b.build(tgt, n_tgt, None, dv)
    assert e.value.status == v.VICP_ERR_OOM
    b.close()
    assert live == {}
