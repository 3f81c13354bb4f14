"""Pins of the oracle's rigid update (Eq. 1): closed-form recovery of a known
transform, numpy's SVD, Horn's quaternion method, the reflection case, the
identity and degenerate geometry."""
import numpy as np
import pytest

import oracle
from paper_2512_04996_gb300.synth import random_rigid


def _horn_rotation(H):
    """Horn (1987): the rotation maximising sum q'.(R p') is the unit
    quaternion of the largest eigenvalue of the symmetric 4x4 built from the
    cross-covariance S = sum p' q'^T."""
    S = H
    N = np.array([
        [S[0, 0] + S[1, 1] + S[2, 2], S[1, 2] - S[2, 1], S[2, 0] - S[0, 2], S[0, 1] - S[1, 0]],
        [S[1, 2] - S[2, 1], S[0, 0] - S[1, 1] - S[2, 2], S[0, 1] + S[1, 0], S[2, 0] + S[0, 2]],
        [S[2, 0] - S[0, 2], S[0, 1] + S[1, 0], -S[0, 0] + S[1, 1] - S[2, 2], S[1, 2] + S[2, 1]],
        [S[0, 1] - S[1, 0], S[2, 0] + S[0, 2], S[1, 2] + S[2, 1], -S[0, 0] - S[1, 1] + S[2, 2]],
    ])
    w, v = np.linalg.eigh(N)
    q0, qx, qy, qz = v[:, np.argmax(w)]
    return np.array([
        [q0 * q0 + qx * qx - qy * qy - qz * qz, 2 * (qx * qy - q0 * qz), 2 * (qx * qz + q0 * qy)],
        [2 * (qy * qx + q0 * qz), q0 * q0 - qx * qx + qy * qy - qz * qz, 2 * (qy * qz - q0 * qx)],
        [2 * (qz * qx - q0 * qy), 2 * (qz * qy + q0 * qx), q0 * q0 - qx * qx - qy * qy + qz * qz],
    ])


def _corr_stats(p, q):
    pb, qb = p.mean(0), q.mean(0)
    return pb, qb, (p - pb).T @ (q - qb)


@pytest.mark.parametrize("seed", range(6))
def test_recovers_known_transform(seed):
    rng = np.random.default_rng(seed)
    T = random_rigid(rng, 170.0, 3.0)
    p = rng.standard_normal((50, 3)) * rng.uniform(0.1, 3, 3)
    q = p @ T[:3, :3].T + T[:3, 3]
    st, dT = oracle.solve(*_corr_stats(p, q))
    assert st == 0
    assert np.abs(dT - T).max() < 1e-12


@pytest.mark.parametrize("seed", range(6))
def test_svd3_matches_numpy(seed):
    rng = np.random.default_rng(20 + seed)
    H = rng.standard_normal((3, 3))
    if seed == 3:
        H[:, 2] = 0.0                                 # rank 2
    U, sig, V = oracle.svd3(H)
    assert np.allclose(sig, np.linalg.svd(H, compute_uv=False), rtol=0, atol=1e-13)
    assert np.allclose(U @ np.diag(sig) @ V.T, H, atol=1e-13)
    assert np.allclose(U.T @ U, np.eye(3), atol=1e-13)
    assert np.allclose(V.T @ V, np.eye(3), atol=1e-13)


@pytest.mark.parametrize("seed", range(6))
def test_rotation_matches_horn(seed):
    rng = np.random.default_rng(40 + seed)
    p = rng.standard_normal((30, 3))
    q = rng.standard_normal((30, 3)) + p @ random_rigid(rng, 90.0, 0.0)[:3, :3].T
    pb, qb, H = _corr_stats(p, q)
    st, dT = oracle.solve(pb, qb, H)
    assert st == 0
    R = dT[:3, :3]
    assert np.allclose(R, _horn_rotation(H), atol=1e-11)
    assert np.allclose(dT[:3, 3], qb - R @ pb, atol=1e-12)


def test_reflection_case_gives_proper_rotation():
    """q is a mirror image of p: the unconstrained orthogonal solution is a
    reflection; Eq. 1 over rotations needs the det fix."""
    rng = np.random.default_rng(9)
    p = rng.standard_normal((40, 3)) * np.array([3.0, 2.0, 0.5])
    q = p * np.array([1.0, 1.0, -1.0])
    pb, qb, H = _corr_stats(p, q)
    U, sig, Vh = np.linalg.svd(H)
    assert np.linalg.det(Vh.T @ U.T) < 0                  # unconstrained optimum reflects
    st, dT = oracle.solve(pb, qb, H)
    R = dT[:3, :3]
    assert st == 0
    assert abs(np.linalg.det(R) - 1.0) < 1e-12
    assert np.allclose(R, _horn_rotation(H), atol=1e-11)
    # and it is the best rotation: no other rotation gives a smaller residual
    res = lambda Rm: (((p - pb) @ Rm.T - (q - qb)) ** 2).sum()
    for s in range(20):
        Rr = random_rigid(np.random.default_rng(s), 180.0, 0.0)[:3, :3]
        assert res(R) <= res(Rr) + 1e-9


def test_identity_gives_zero_update():
    rng = np.random.default_rng(1)
    p = rng.standard_normal((100, 3))
    st, dT = oracle.solve(*_corr_stats(p, p.copy()))
    assert st == 0 and np.abs(dT - np.eye(4)).max() < 1e-14


def test_degenerate_geometry():
    rng = np.random.default_rng(2)
    line = np.outer(rng.standard_normal(50), [1.0, 2.0, -0.5])
    st, _ = oracle.solve(*_corr_stats(line, line + 0.3))
    assert st == oracle.ERR_DEGENERATE
    st, _ = oracle.solve(np.zeros(3), np.zeros(3), np.zeros((3, 3)))
    assert st == oracle.ERR_DEGENERATE
    plane = np.column_stack([rng.standard_normal((50, 2)), np.zeros(50)])
    st, _ = oracle.solve(*_corr_stats(plane, plane))     # rank 2 is solvable
    assert st == 0


def test_compose_is_matrix_product():
    rng = np.random.default_rng(3)
    A, B = random_rigid(rng, 30, 1), random_rigid(rng, 30, 1)
    assert np.allclose(oracle.compose(A, B), A @ B, atol=1e-15)
