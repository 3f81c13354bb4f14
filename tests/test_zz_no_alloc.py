"""vicp_offsets_static (voxel keys and offsets in the library's static
scratch, no device allocation) against vicp_build_grid + vicp_get_grid on the
same grid: bit-exact keys and offsets on consecutive calls with different
clouds and grid sizes, device memory unchanged by calls after the first, and
the size and argument checks.  Collected last so that it also runs after every
other GPU test in one process."""
import gc

import numpy as np
import pytest
import torch

import oracle
from gpu_util import context, to_np, vicp

pytestmark = pytest.mark.gpu


def _expected(target, origin=None, voxel_size=0.0, dims=None, divisions=64):
    """Keys, offsets and the grid from the context entry point."""
    ctx = context(L=0, voxel_size=voxel_size, divisions=divisions, origin=origin, dims=dims)
    ctx.build_grid(target)
    g = ctx.get_grid()
    out = dict(keys=to_np(g["keys"]).copy(), offsets=to_np(g["offsets"]).copy(),
               origin=tuple(float(x) for x in g["origin"]), voxel_size=float(g["voxel_size"]),
               dims=tuple(int(x) for x in g["dims"]))
    ctx.close()
    return out


def _run_static(v, target, e, keys, offsets):
    v.vicp_offsets_static(target, e["origin"], e["voxel_size"], e["dims"], keys, offsets)
    torch.cuda.synchronize()
    V = int(np.prod(e["dims"]))
    return to_np(keys), to_np(offsets[:V + 1]).view(np.uint32)


def test_static_offsets_equal_build_grid_on_consecutive_calls(pairs):
    v = vicp()
    scene = torch.from_numpy(pairs(3).target).cuda()          # 226k points, ~10.9M voxels
    sp = pairs(1)
    small = torch.from_numpy(sp.target).cuda()
    lo = sp.target[:, :3].min(0)
    # an explicit grid that leaves part of the cloud outside (keys -1)
    e_small = _expected(small, origin=lo + 0.2, voxel_size=0.041, dims=(37, 29, 41))
    e_scene = _expected(scene, voxel_size=pairs(3).voxel_size)
    assert (e_small["keys"] < 0).any() and (e_small["keys"] >= 0).any()
    assert int(np.prod(e_scene["dims"])) <= v.VICP_STATIC_MAX_VOXELS

    torch.cuda.synchronize()
    k_scene = torch.empty(scene.shape[0], dtype=torch.int32, device="cuda")
    o_scene = torch.empty(int(np.prod(e_scene["dims"])) + 1, dtype=torch.int32, device="cuda")
    k_small = torch.empty(small.shape[0], dtype=torch.int32, device="cuda")
    o_small = torch.empty(int(np.prod(e_small["dims"])) + 1, dtype=torch.int32, device="cuda")

    # first call (looks up the scratch address on this device)
    keys, off = _run_static(v, scene, e_scene, k_scene, o_scene)
    assert np.array_equal(keys, e_scene["keys"]) and np.array_equal(off, e_scene["offsets"])
    # and directly against the oracle's keys and offsets on the same grid
    g = oracle.explicit_grid(e_scene["origin"], e_scene["voxel_size"], e_scene["dims"])
    rkeys = oracle.keys(g, pairs(3).target)
    assert np.array_equal(keys, rkeys)
    assert np.array_equal(off, oracle.offsets(oracle.histogram(rkeys, g.n_voxels)))

    # device memory must not move across the next calls: objects of earlier
    # tests that hold device buffers are collected first, and the collector
    # is held off meanwhile (a context freed mid-test raised the free count)
    gc.collect()
    torch.cuda.synchronize()
    gc.disable()
    try:
        free0 = torch.cuda.mem_get_info()[0]
        keys, off = _run_static(v, small, e_small, k_small, o_small)   # smaller grid after a larger one
        assert np.array_equal(keys, e_small["keys"]) and np.array_equal(off, e_small["offsets"])
        keys, off = _run_static(v, scene, e_scene, k_scene, o_scene)   # and back: scratch cleared each call
        assert np.array_equal(keys, e_scene["keys"]) and np.array_equal(off, e_scene["offsets"])
        assert torch.cuda.mem_get_info()[0] == free0
    finally:
        gc.enable()


def test_static_offsets_repeat_same_input(pairs):
    v = vicp()
    p = pairs(2)
    t = torch.from_numpy(p.target).cuda()
    e = _expected(t, voxel_size=p.voxel_size, divisions=p.grid_divisions)
    k = torch.empty(t.shape[0], dtype=torch.int32, device="cuda")
    o = torch.empty(int(np.prod(e["dims"])) + 1, dtype=torch.int32, device="cuda")
    for _ in range(2):
        keys, off = _run_static(v, t, e, k, o)
        assert np.array_equal(keys, e["keys"]) and np.array_equal(off, e["offsets"])


def _raw(v, t, origin, h, dims, keys, offsets):
    """The C entry point itself, with no checks in between."""
    import ctypes as C
    lib = v.load_library()
    o = (C.c_float * 3)(*origin)
    d = (C.c_int32 * 3)(*dims)
    return lib.vicp_offsets_static(C.c_void_p(t.data_ptr()), t.shape[0], o, h, d, C.c_void_p(keys.data_ptr()),
                                   C.c_void_p(offsets.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_static_offsets_rejects_large_grids_and_bad_arguments():
    v = vicp()
    t = torch.zeros((64, 4), dtype=torch.float32, device="cuda")
    k = torch.empty(64, dtype=torch.int32, device="cuda")
    o = torch.empty(4096 + 8, dtype=torch.int32, device="cuda")
    # too many voxels; too many brick slots (checked before any launch)
    for dims in ((257, 256, 256), (1, 1, 1 << 21)):
        assert _raw(v, t, (0.0, 0.0, 0.0), 1.0, dims, k, o) == v.VICP_ERR_GRID_TOO_LARGE
    with pytest.raises(v.VicpError) as err:
        v.vicp_offsets_static(t, (0.0, 0.0, 0.0), 1.0, (4096, 4096, 2))
    assert err.value.status == v.VICP_ERR_GRID_TOO_LARGE
    for origin, h, dims in (((0.0, 0.0, 0.0), 0.0, (16, 16, 16)), ((0.0, 0.0, 0.0), float("nan"), (16, 16, 16)),
                            ((0.0, 0.0, 0.0), 1.0, (0, 4, 4)), ((float("inf"), 0.0, 0.0), 1.0, (16, 16, 16))):
        assert _raw(v, t, origin, h, dims, k, o) == v.VICP_ERR_INVALID
    # offsets not 16-byte aligned; keys not 4-byte aligned
    assert _raw(v, t, (0.0, 0.0, 0.0), 1.0, (16, 16, 16), k, o[1:]) == v.VICP_ERR_INVALID
    kb = k.view(torch.uint8)[1:]
    assert _raw(v, t, (0.0, 0.0, 0.0), 1.0, (16, 16, 16), kb, o) == v.VICP_ERR_INVALID
    # a valid call still works afterwards
    v.vicp_offsets_static(t, (0.0, 0.0, 0.0), 1.0, (16, 16, 16), k, o)
    torch.cuda.synchronize()
    assert np.array_equal(to_np(k), np.zeros(64, np.int32))
    off = to_np(o[:4097])
    assert off[0] == 0 and np.all(off[1:] == 64)
