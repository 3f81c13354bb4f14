"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and bring its arrays back as numpy, and compare them with the oracle's."""
import numpy as np
import torch

import oracle


def vicp():
    from paper_2512_04996_gb300 import vicp as v
    v.load_library(build_if_missing=True)
    return v


def to_np(t):
    if not torch.is_tensor(t):
        return t
    if t.dtype == torch.uint32:
        return t.view(torch.int32).cpu().numpy().view(np.uint32)
    return t.cpu().numpy()


def context(L=10, voxel_size=0.0, divisions=64, origin=None, dims=None, flags=0, max_iters=30, eps=0.0):
    v = vicp()
    kw = dict(voxel_size=float(voxel_size), grid_divisions=int(divisions), dilation_layers=int(L),
              flags=int(flags), max_iters=int(max_iters), rmse_eps=float(eps))
    if dims is not None:
        kw.update(origin=tuple(origin), dims=tuple(dims))
    return v.Context(**kw)


def gpu_grid(target, L=10, **kw):
    """Build + dilate on the GPU; returns (ctx, dict of numpy arrays)."""
    ctx = context(L=L, **kw)
    t = torch.from_numpy(np.ascontiguousarray(target)).cuda()
    ctx.build_grid(t)
    ctx.dilate(L)
    g = {k: to_np(v) for k, v in ctx.get_grid().items()}
    g["_target"] = t
    return ctx, g


def oracle_grid_for(g_gpu, target, L):
    """The oracle's build on the geometry the GPU reported."""
    grid = oracle.Grid(g_gpu["origin"], g_gpu["voxel_size"], g_gpu["inv_voxel_size"], g_gpu["dims"])
    return grid, oracle.build_grid(grid, target, L)


def assert_grid_equal(g, ref, target):
    """Keys, offsets, occupancy, root and ring bit-exact; each CSR segment the
    same set of point indices (the order inside a segment is unspecified)."""
    V = g["n_voxels"]
    assert np.array_equal(g["keys"], ref["keys"])
    assert np.array_equal(g["offsets"], ref["off"])
    assert g["n_stored"] == int(ref["off"][-1])
    counts = np.diff(ref["off"].astype(np.int64))
    seg = np.repeat(np.arange(V), counts)
    ids = g["ids"]
    assert np.array_equal(ids[np.lexsort((ids, seg))], ref["ids"])
    pts = g["csr_points"]
    assert np.array_equal(pts[:, :3], target[ids, :3])
    assert np.array_equal(pts[:, 3].view(np.int32), ids)
    bits = np.unpackbits(g["occupancy"].view(np.uint8), bitorder="little")[:V]
    assert np.array_equal(bits.astype(bool), counts > 0)
    if "root" in g:
        assert np.array_equal(g["root"], ref["root"])
        assert np.array_equal(g["ring"], ref["ring"])


def transform_f32(T, pts):
    """s_a = ((R_a0*x + R_a1*y) + R_a2*z) + t_a in float32, one rounding per op."""
    R = T[:3, :3].astype(np.float32)
    t = T[:3, 3].astype(np.float32)
    out = np.zeros((pts.shape[0], 4), np.float32)
    for a in range(3):
        acc = R[a, 0] * pts[:, 0]
        acc = acc + R[a, 1] * pts[:, 1]
        acc = acc + R[a, 2] * pts[:, 2]
        out[:, a] = acc + t[a]
    return out


def rot_err(Ta, Tb):
    E = Ta[:3, :3] @ Tb[:3, :3].T
    return float(np.arccos(np.clip((np.trace(E) - 1.0) / 2.0, -1.0, 1.0)))
