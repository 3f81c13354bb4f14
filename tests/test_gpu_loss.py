"""The differentiable loss on the GPU (vicp_se3_exp, vicp_se3_left_jacobian_t,
vicp_batch_loss and the autograd Function) against the oracle (oracle/diff.py):
the SE(3) maps to FP64 rounding, the loss and its analytic gradients with the
GPU's correspondences, and the gradients against FP64 central finite
differences (h = 1e-4, correspondences frozen) at relative error <= 1e-4,
measured against the gradient's largest component."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import assert_nn_equal, to_np, vicp
from oracle import diff
from paper_2512_04996_gb300 import synth

pytestmark = pytest.mark.gpu

L = 10
FD_TOL = 1e-4


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


def _xi(rng, angle, trans=0.05):
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    return np.concatenate([rng.normal(size=3) * trans, axis * angle])


def test_se3_maps_match_oracle():
    v = vicp()
    rng = np.random.default_rng(1)
    angles = [0.0, 1e-9, 5e-5, 2e-4, 0.01, 0.3, 1.0, 1.99, 2.01, 3.1]
    xi = np.stack([_xi(rng, a, 0.7) for a in angles])
    T0 = np.stack([diff.se3_exp(_xi(rng, 0.5, 0.3)) for _ in angles])
    g = rng.normal(size=(len(angles), 6))
    xd = torch.from_numpy(xi).cuda()
    T = to_np(v.vicp_se3_exp(xd, torch.from_numpy(T0).cuda()))
    out = to_np(v.vicp_se3_left_jacobian_t(xd, torch.from_numpy(g).cuda()))
    for k in range(len(angles)):
        assert np.allclose(T[k], diff.se3_exp(xi[k]) @ T0[k], rtol=0, atol=1e-14)
        ref = diff.se3_left_jacobian(xi[k]).T @ g[k]
        assert np.allclose(out[k], ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def _setup(ps, poses):
    v = vicp()
    tgt = np.ascontiguousarray(np.concatenate([p.target for p in ps]))
    src = np.ascontiguousarray(np.concatenate([p.source for p in ps]))
    n_tgt = np.array([p.target.shape[0] for p in ps], np.int32)
    n_src = np.array([p.source.shape[0] for p in ps], np.int32)
    b = v.Batch(dilation_layers=L)
    t = torch.from_numpy(tgt).cuda()
    b.build(t, n_tgt, None, np.array([p.grid_divisions for p in ps], np.int32))
    s = torch.from_numpy(src).cuda()
    T = torch.from_numpy(np.ascontiguousarray(poses)).cuda()
    nn, d2 = b.correspond(s, n_src, T)
    return v, b, t, s, n_src, T, to_np(nn), to_np(d2)


def _split(a, n_src):
    return np.split(a, np.cumsum(n_src)[:-1])


@pytest.fixture(scope="module")
def loss_pairs():
    return synth.loss_pairs(n_pairs=6)


@pytest.mark.parametrize("where", ["truth", "identity"])
def test_loss_and_analytic_gradients_match_oracle(loss_pairs, where):
    ps = loss_pairs
    rng = np.random.default_rng(2)
    poses = np.stack([diff.se3_exp(_xi(rng, 0.01, 0.005)) @ p.T_gt if where == "truth" else np.eye(4)
                      for p in ps])
    v, b, t, s, n_src, T, nn, d2 = _setup(ps, poses)
    loss, gp, gs = b.loss(s, n_src, T, torch.from_numpy(nn).cuda(), grad_pose=True, grad_src=True)
    loss, gp, gs = to_np(loss), to_np(gp), to_np(gs)
    nn_k, gs_k, d2_k = _split(nn, n_src), _split(gs, n_src), _split(d2, n_src)
    for k, p in enumerate(ps):
        # the search itself against the oracle, every pair
        og = oracle.fit_grid(p.target, 0.0, p.grid_divisions)
        rnn, rd2, _ = oracle.correspond(og, oracle.build_grid(og, p.target, L), p.target, p.source, poses[k])
        assert_nn_equal(nn_k[k], d2_k[k], rnn, rd2)
        ref = diff.loss(p.target, p.source, poses[k], nn_k[k])
        assert abs(loss[k] - ref) <= 1e-12 * ref
        assert _rel(gp[k], diff.grad_left(p.target, p.source, poses[k], nn_k[k])) <= 1e-9
        gref = diff.grad_points(p.target, p.source, poses[k], nn_k[k])
        assert np.abs(gs_k[k][:, :3] - gref).max() <= 2e-6 * np.abs(gref).max()
        assert np.all(gs_k[k][:, 3] == 0.0)


@pytest.mark.parametrize("angle", [0.0, 0.05, 0.4])
def test_autograd_gradients_pass_the_finite_difference_check(loss_pairs, angle):
    """dL/dxi through the autograd Function at xi (zero, or a rotation of
    `angle`) against FP64 central differences of the oracle's loss with the
    GPU's correspondences frozen (h = 1e-4); dL/dp for sampled points too."""
    ps = loss_pairs
    rng = np.random.default_rng(3)
    T0 = np.stack([diff.se3_exp(_xi(rng, 0.02, 0.01)) @ p.T_gt for p in ps])
    xi = np.stack([_xi(rng, angle, 0.02) if angle else np.zeros(6) for _ in ps])
    T = np.stack([diff.se3_exp(xi[k]) @ T0[k] for k in range(len(ps))])
    v, b, t, s, n_src, Td, nn, _ = _setup(ps, T)
    xi_t = torch.from_numpy(xi).cuda().requires_grad_(True)
    src_t = s.clone().requires_grad_(True)
    loss = v.point_to_point_loss(xi_t, src_t, b, n_src, torch.from_numpy(np.ascontiguousarray(T0)).cuda())
    w = torch.linspace(0.5, 1.5, len(ps), dtype=torch.float64, device="cuda")
    (loss * w).sum().backward()
    gx, gs = to_np(xi_t.grad), to_np(src_t.grad)
    nn_k, gs_k = _split(nn, n_src), _split(gs, n_src)
    wk = to_np(w)
    for k, p in enumerate(ps):
        fd = diff.fd_xi(xi[k], T0[k], p.target, p.source, nn_k[k], h=1e-4)
        assert _rel(gx[k], wk[k] * fd) <= FD_TOL, (k, gx[k], wk[k] * fd)
        idx = np.random.default_rng(k).choice(p.source.shape[0], 4, replace=False)
        fdp = diff.fd_points(idx, p.target, p.source, T[k], nn_k[k], h=1e-4)
        assert _rel(gs_k[k][idx, :3], wk[k] * fdp) <= FD_TOL


def test_recomputed_correspondences_give_identical_gradients(loss_pairs):
    ps = loss_pairs[:3]
    rng = np.random.default_rng(4)
    T0 = np.ascontiguousarray(np.stack([diff.se3_exp(_xi(rng, 0.02, 0.01)) @ p.T_gt for p in ps]))
    v, b, t, s, n_src, Td, nn, _ = _setup(ps, T0)
    grads = []
    for recompute in (False, True):
        xi_t = torch.zeros((len(ps), 6), dtype=torch.float64, device="cuda", requires_grad=True)
        src_t = s.clone().requires_grad_(True)
        loss = v.point_to_point_loss(xi_t, src_t, b, n_src, torch.from_numpy(T0).cuda(), recompute)
        loss.sum().backward()
        grads.append((to_np(loss.detach()), to_np(xi_t.grad), to_np(src_t.grad)))
    for a, c in zip(grads[0], grads[1]):
        assert np.array_equal(a, c)


def test_float32_parameters(loss_pairs):
    """xi given in float32 (6 fp32 parameters per pair) gets a float32
    gradient equal to the float64 one rounded."""
    ps = loss_pairs[:2]
    T0 = np.ascontiguousarray(np.stack([p.T_gt for p in ps]))
    v, b, t, s, n_src, Td, nn, _ = _setup(ps, T0)
    out = []
    for dt in (torch.float64, torch.float32):
        xi_t = torch.zeros((len(ps), 6), dtype=dt, device="cuda", requires_grad=True)
        v.point_to_point_loss(xi_t, s, b, n_src, torch.from_numpy(T0).cuda()).sum().backward()
        out.append(to_np(xi_t.grad))
    assert out[1].dtype == np.float32 and np.array_equal(out[1], out[0].astype(np.float32))


def test_full_loss_workload_sampled():
    """The 64-pair, 20k-point workload: loss and gradients of all pairs on the
    GPU; the oracle checks every eighth pair (analytic values) and two pairs
    by finite differences."""
    ps = synth.loss_pairs()
    assert len(ps) == 64
    rng = np.random.default_rng(6)
    T0 = np.ascontiguousarray(np.stack([diff.se3_exp(_xi(rng, 0.02, 0.01)) @ p.T_gt for p in ps]))
    v, b, t, s, n_src, Td, nn, _ = _setup(ps, T0)
    xi_t = torch.zeros((64, 6), dtype=torch.float32, device="cuda", requires_grad=True)
    loss = v.point_to_point_loss(xi_t, s, b, n_src, torch.from_numpy(T0).cuda())
    loss.sum().backward()
    loss, gx = to_np(loss.detach()), to_np(xi_t.grad).astype(np.float64)
    nn_k = _split(nn, n_src)
    for k in range(0, 64, 8):
        p = ps[k]
        assert abs(loss[k] - diff.loss(p.target, p.source, T0[k], nn_k[k])) <= 1e-12 * loss[k]
        g = diff.grad_left(p.target, p.source, T0[k], nn_k[k])
        assert _rel(gx[k], g) <= 1e-6   # float32 parameters
    for k in (5, 40):
        p = ps[k]
        fd = diff.fd_xi(np.zeros(6), T0[k], p.target, p.source, nn_k[k], h=1e-4)
        assert _rel(gx[k], fd) <= FD_TOL
