"""Pins of the oracle's differentiable loss (oracle/diff.py): the SE(3)
exponential against scipy's matrix exponential of the twist, the left
Jacobian against a numerical derivative through scipy's matrix logarithm,
the series branches against the closed forms on both sides of their
thresholds, and every gradient against central finite differences with the
correspondences held fixed (FP64, h = 1e-4), plus the translation-only
closed form."""
import numpy as np
import pytest
from scipy.linalg import expm, logm

from oracle import diff

ANGLES = [0.0, 1e-9, 9.9e-5, 1.01e-4, 1e-3, 0.05, 0.3, 1.0, 1.999, 2.001, 3.0]


def _twist(xi):
    X = np.zeros((4, 4))
    X[:3, :3] = diff.hat(xi[3:])
    X[:3, 3] = xi[:3]
    return X


def _vee(X):
    return np.array([X[0, 3], X[1, 3], X[2, 3], X[2, 1], X[0, 2], X[1, 0]])


def _xi(rng, angle):
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    return np.concatenate([rng.normal(size=3) * 0.7, axis * angle])


@pytest.mark.parametrize("angle", ANGLES)
def test_exp_is_the_matrix_exponential_of_the_twist(angle):
    rng = np.random.default_rng(int(angle * 1e4) + 1)
    xi = _xi(rng, angle)
    assert np.allclose(diff.se3_exp(xi), expm(_twist(xi)), rtol=0, atol=2e-15)
    assert np.allclose(diff.se3_exp(xi) @ diff.se3_exp(-xi), np.eye(4), rtol=0, atol=4e-15)


@pytest.mark.parametrize("angle", ANGLES)
def test_left_jacobian_is_the_derivative_of_exp(angle):
    """Exp(xi + e) Exp(xi)^-1 = Exp(J(xi) e) + O(e^2): the central difference
    of its logarithm in e gives J(xi) column by column."""
    rng = np.random.default_rng(int(angle * 1e4) + 7)
    xi = _xi(rng, angle)
    J = diff.se3_left_jacobian(xi)
    E0inv = np.linalg.inv(expm(_twist(xi)))
    eps = 1e-6
    num = np.zeros((6, 6))
    for k in range(6):
        e = np.zeros(6)
        e[k] = eps
        lp = _vee(np.real(logm(expm(_twist(xi + e)) @ E0inv)))
        lm = _vee(np.real(logm(expm(_twist(xi - e)) @ E0inv)))
        num[:, k] = (lp - lm) / (2 * eps)
    assert np.allclose(J, num, rtol=0, atol=2e-8), np.abs(J - num).max()


def test_left_jacobian_at_zero_is_identity_and_blocks():
    assert np.array_equal(diff.se3_left_jacobian(np.zeros(6)), np.eye(6))
    rng = np.random.default_rng(3)
    xi = _xi(rng, 0.8)
    J = diff.se3_left_jacobian(xi)
    assert np.array_equal(J[3:, :3], np.zeros((3, 3)))
    assert np.allclose(J[:3, :3], J[3:, 3:])
    # the SO(3) block: Exp(phi + e) Exp(phi)^T = Exp(J e) to first order
    assert np.allclose(J[:3, :3], diff.so3_left_jacobian(xi[3:]))


@pytest.mark.parametrize("t", [1e-4, 2.0])
def test_series_meet_the_closed_forms_at_their_thresholds(t):
    """Each coefficient to 1e-14 relative on both sides of the branch points
    and elsewhere, against the closed forms in 40-digit arithmetic."""
    import mpmath as mp
    mp.mp.dps = 40
    for x in (t * (1 - 1e-9), t * (1 + 1e-9), 0.3 * t, 0.7 * t, 1.5 * t):
        X = mp.mpf(x)
        ref = [mp.sin(X) / X, (1 - mp.cos(X)) / X ** 2, (X - mp.sin(X)) / X ** 3,
               (X ** 2 / 2 + mp.cos(X) - 1) / X ** 4, (X - mp.sin(X) - X ** 3 / 6) / X ** 5]
        for got, r in zip(diff._coeffs(x), ref):
            assert abs(got - float(r)) <= 1e-14 * abs(float(r)), (x, got, float(r))


def _problem(seed, m=300, n=500):
    rng = np.random.default_rng(seed)
    tgt = np.zeros((n, 4), np.float32)
    tgt[:, :3] = rng.normal(size=(n, 3))
    src = np.zeros((m, 4), np.float32)
    src[:, :3] = rng.normal(size=(m, 3))
    nn = rng.integers(0, n, m).astype(np.int32)
    T0 = diff.se3_exp(_xi(rng, 0.6))
    return tgt, src, nn, T0


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_pose_gradient_at_zero_matches_finite_differences():
    tgt, src, nn, T0 = _problem(11)
    g = diff.grad_left(tgt, src, T0, nn)
    assert _rel(g, diff.fd_xi(np.zeros(6), T0, tgt, src, nn)) <= 1e-6
    assert np.array_equal(diff.grad_xi(np.zeros(6), T0, tgt, src, nn), g)


@pytest.mark.parametrize("angle", [1e-3, 0.2, 0.45, 1.3])
def test_pose_gradient_away_from_zero_matches_finite_differences(angle):
    tgt, src, nn, T0 = _problem(13)
    xi = _xi(np.random.default_rng(5), angle)
    assert _rel(diff.grad_xi(xi, T0, tgt, src, nn), diff.fd_xi(xi, T0, tgt, src, nn)) <= 1e-6


def test_point_gradient_matches_finite_differences():
    tgt, src, nn, T0 = _problem(17)
    idx = [0, 5, 77, 299]
    g = diff.grad_points(tgt, src, T0, nn)[idx]
    assert _rel(g, diff.fd_points(idx, tgt, src, T0, nn)) <= 1e-6


def test_translation_only_closed_form():
    """With T = translation by rho only, L = mean |p + rho - q|^2 and
    dL/drho = 2 mean(p + rho - q)."""
    tgt, src, nn, _ = _problem(19)
    rho = np.array([0.3, -0.2, 0.1])
    T = np.eye(4)
    T[:3, 3] = rho
    p = src[:, :3].astype(np.float64)
    q = tgt[nn, :3].astype(np.float64)
    assert np.isclose(diff.loss(tgt, src, T, nn), np.mean(np.sum((p + rho - q) ** 2, axis=1)), rtol=1e-15)
    assert np.allclose(diff.grad_left(tgt, src, T, nn)[:3], 2 * np.mean(p + rho - q, axis=0), rtol=1e-14)
