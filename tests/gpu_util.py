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
    """Angle (rad) of the rotation between two poses, from the Frobenius norm
    of the difference of their rotations (|Ra - Rb|_F = 2 sqrt(2) sin(a/2)),
    which keeps full relative precision for small angles where the arccos of
    the trace cannot resolve less than about 1e-8 rad."""
    d = np.linalg.norm(np.asarray(Ta)[:3, :3] - np.asarray(Tb)[:3, :3])
    return float(2.0 * np.arcsin(min(1.0, d / (2.0 * np.sqrt(2.0)))))


def assert_nn_equal(nn, d2, rnn, rd2):
    """Each neighbour equals the oracle's; another index is allowed only when
    its float squared distance is within 1e-6 relative of the oracle's.
    Where the indices agree, the squared distances agree bit for bit."""
    nn, d2, rnn, rd2 = (np.asarray(x) for x in (nn, d2, rnn, rd2))
    assert nn.shape == rnn.shape
    same = nn == rnn
    if not same.all():
        bad = ~same
        rel = np.abs(d2[bad].astype(np.float64) - rd2[bad]) / np.maximum(rd2[bad], 1e-30)
        assert (rel <= 1e-6).all(), (np.flatnonzero(bad)[:5], nn[bad][:5], rnn[bad][:5])
    both_nan = np.isnan(d2) & np.isnan(rd2)
    assert np.array_equal(d2[same & ~both_nan], rd2[same & ~both_nan])
