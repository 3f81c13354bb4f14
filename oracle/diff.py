"""CPU oracle of the differentiable point-to-point loss -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may import this module.  Plain numpy in FP64, written from the definitions:

* the loss of one pair is the mean squared point-to-point residual of Eq. 1,
  L = (1/M) sum_i |T p_i - q_nn(i)|^2, with the correspondences nn held
  fixed (they come from the NNS of Alg. 4 and carry no gradient);
* poses are perturbed on the left in se(3): T(xi) = Exp(xi) T0 with
  xi = (rho, phi) (translation part first, rotation part second) and Exp the
  SE(3) exponential, the matrix exponential of the 4x4 twist
  [[phi^, rho], [0, 0]];
* the left-perturbation gradient at T is the gradient of L(Exp(d) T) in d
  at d = 0: (2/M) (sum r_i, sum s_i x r_i) with s_i = T p_i and
  r_i = s_i - q_i; the gradient in xi at any xi is J(xi)^T times it, with
  J the left Jacobian of SE(3), Exp(xi + e) = Exp(J(xi) e) Exp(xi) + O(e^2);
* the gradient in a source point is (2/M) R^T r_i.

The closed forms of Exp and J follow the standard series of the SE(3)
exponential (Rodrigues' formula for the rotation block and the series of
its left Jacobians); small angles use their Taylor polynomials.
"""
from __future__ import annotations

import numpy as np


def hat(w) -> np.ndarray:
    """The skew matrix w^ with w^ x = w cross x."""
    x, y, z = (float(v) for v in w)
    return np.array([[0.0, -z, y], [z, 0.0, -x], [-y, x, 0.0]])


def _series(t2: float, first: int, sign: float) -> float:
    """sum_k sign (-1)^k t^(2k) / (2k + first)!, to full FP64 precision."""
    term = sign
    for j in range(2, first + 1):
        term /= j
    total = term
    k = 0
    while abs(term) > 1e-20 * abs(total) and k < 40:
        k += 1
        term *= -t2 / ((2 * k + first - 1) * (2 * k + first))
        total += term
    return total


def _coeffs(theta: float):
    """a = sin(t)/t, b = (1 - cos t)/t^2, c = (t - sin t)/t^3,
    d = (t^2/2 + cos t - 1)/t^4, e = (t - sin t - t^3/6)/t^5.  b is taken as
    2 sin^2(t/2)/t^2 (no cancellation).  c, d and e cancel in closed form at
    small t, so for t < 2 each is its Taylor series summed to full
    precision: c = sum (-1)^k t^2k/(2k+3)!, d = sum (-1)^k t^2k/(2k+4)!,
    e = -sum (-1)^k t^2k/(2k+5)!."""
    t = float(theta)
    t2 = t * t
    if t < 1e-4:
        a = 1.0 - t2 / 6.0 + t2 * t2 / 120.0
        b = 0.5 - t2 / 24.0 + t2 * t2 / 720.0
    else:
        a = np.sin(t) / t
        b = 2.0 * (np.sin(0.5 * t) / t) ** 2
    if t < 2.0:
        c, d, e = _series(t2, 3, 1.0), _series(t2, 4, 1.0), _series(t2, 5, -1.0)
    else:
        c = (t - np.sin(t)) / t ** 3
        d = (t2 / 2.0 + np.cos(t) - 1.0) / t ** 4
        e = (t - np.sin(t) - t ** 3 / 6.0) / t ** 5
    return a, b, c, d, e


def so3_exp(phi) -> np.ndarray:
    """Rodrigues: I + a phi^ + b phi^2."""
    th = float(np.linalg.norm(phi))
    a, b, *_ = _coeffs(th)
    P = hat(phi)
    return np.eye(3) + a * P + b * (P @ P)


def so3_left_jacobian(phi) -> np.ndarray:
    """I + b phi^ + c phi^2."""
    th = float(np.linalg.norm(phi))
    _, b, c, *_ = _coeffs(th)
    P = hat(phi)
    return np.eye(3) + b * P + c * (P @ P)


def se3_exp(xi) -> np.ndarray:
    """Exp(xi) for xi = (rho, phi): [[so3_exp(phi), J(phi) rho], [0, 1]]."""
    xi = np.asarray(xi, dtype=np.float64)
    T = np.eye(4)
    T[:3, :3] = so3_exp(xi[3:])
    T[:3, 3] = so3_left_jacobian(xi[3:]) @ xi[:3]
    return T


def se3_left_jacobian(xi) -> np.ndarray:
    """The 6x6 left Jacobian [[J, Q], [0, J]] of SE(3) at xi = (rho, phi),
    J the left Jacobian of SO(3) at phi and
    Q = rho^/2 + c (P R + R P + P R P) + d (P P R + R P P - 3 P R P)
        + (d + 3 e)/2 (P R P P + P P R P),   P = phi^, R = rho^."""
    xi = np.asarray(xi, dtype=np.float64)
    rho, phi = xi[:3], xi[3:]
    th = float(np.linalg.norm(phi))
    _, _, c, d, e = _coeffs(th)
    P, R = hat(phi), hat(rho)
    Q = (0.5 * R + c * (P @ R + R @ P + P @ R @ P) + d * (P @ P @ R + R @ P @ P - 3.0 * P @ R @ P)
         + 0.5 * (d + 3.0 * e) * (P @ R @ P @ P + P @ P @ R @ P))
    J = so3_left_jacobian(phi)
    out = np.zeros((6, 6))
    out[:3, :3] = J
    out[:3, 3:] = Q
    out[3:, 3:] = J
    return out


def residuals(target, source, T, nn) -> tuple[np.ndarray, np.ndarray]:
    """s_i = T p_i and r_i = s_i - q_nn(i), in FP64."""
    p = np.asarray(source, dtype=np.float64)[:, :3]
    q = np.asarray(target, dtype=np.float64)[np.asarray(nn), :3]
    s = p @ T[:3, :3].T + T[:3, 3]
    return s, s - q


def loss(target, source, T, nn) -> float:
    """(1/M) sum_i |T p_i - q_nn(i)|^2."""
    _, r = residuals(target, source, T, nn)
    return float(np.mean(np.sum(r * r, axis=1)))


def grad_left(target, source, T, nn) -> np.ndarray:
    """Left-perturbation gradient (2/M) (sum r_i, sum s_i x r_i)."""
    s, r = residuals(target, source, T, nn)
    M = s.shape[0]
    return np.concatenate([2.0 / M * r.sum(0), 2.0 / M * np.cross(s, r).sum(0)])


def grad_points(target, source, T, nn) -> np.ndarray:
    """(2/M) R^T r_i per source point, (M, 3)."""
    _, r = residuals(target, source, T, nn)
    return 2.0 / r.shape[0] * (r @ T[:3, :3])


def grad_xi(xi, T0, target, source, nn) -> np.ndarray:
    """dL/dxi of L(Exp(xi) T0) with fixed correspondences."""
    T = se3_exp(xi) @ T0
    return se3_left_jacobian(xi).T @ grad_left(target, source, T, nn)


def fd_xi(xi, T0, target, source, nn, h: float = 1e-4) -> np.ndarray:
    """Central finite differences of L(Exp(xi) T0) in each xi_k, step h."""
    xi = np.asarray(xi, dtype=np.float64)
    g = np.zeros(6)
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        g[k] = (loss(target, source, se3_exp(xi + e) @ T0, nn) - loss(target, source, se3_exp(xi - e) @ T0, nn)) \
            / (2.0 * h)
    return g


def fd_points(idx, target, source, T, nn, h: float = 1e-4) -> np.ndarray:
    """Central finite differences of L in the coordinates of source points
    idx, (len(idx), 3)."""
    src = np.asarray(source, dtype=np.float64).copy()
    out = np.zeros((len(idx), 3))
    for n, i in enumerate(idx):
        for a in range(3):
            keep = src[i, a]
            src[i, a] = keep + h
            lp = loss(target, src, T, nn)
            src[i, a] = keep - h
            lm = loss(target, src, T, nn)
            src[i, a] = keep
            out[n, a] = (lp - lm) / (2.0 * h)
    return out
