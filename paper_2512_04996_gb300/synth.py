"""Seeded synthetic point-cloud pairs shaped like the paper's workloads.

The paper evaluates on ModelNet objects (~10k points), the Stanford Bunny
(~40k points) and TUM RGB-D scenes (~226k points), all normalised to the unit
sphere and perturbed by a random rigid motion (Sec. 4.1, "Dataset").  None of
those datasets ships with this repository, so these generators stand in for
their size and structure:

* ``sphere_plane``  -- 4,096 points: unit sphere plus a 1x1 plane.
* ``bumpy_object``  -- 40,000 points on a closed bumpy surface with a 10:1
  sampling-density gradient (object scale, Bunny-sized).
* ``depth_scene``   -- ~226,000 points back-projected from a synthetic 640x480
  depth image of planes and boxes (scene scale, TUM-sized).
* ``batched_pairs`` -- many independent pairs of uneven sizes.

This module holds no arithmetic of the registration method itself (no
voxelisation, no nearest-neighbour search, no pose solve).  It only draws
random clouds and applies the ground-truth rigid motion that the method is
later asked to recover.  Both the CUDA path and the CPU oracle receive the
arrays it returns as plain inputs.

Every cloud is returned as a C-contiguous ``float32`` array of shape (N, 4)
with ``w = 0``: the fourth lane pads each point to 16 bytes.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

__all__ = [
    "Pair",
    "random_rigid",
    "sphere_plane",
    "bumpy_object",
    "depth_scene",
    "batched_pairs",
    "make_config",
    "CONFIG_SEEDS",
]

# One fixed seed per workload, so every run of tests and benchmarks sees the
# same clouds.
CONFIG_SEEDS = {1: 1001, 2: 1002, 3: 1003, 4: 1004, 5: 1005}


@dataclass
class Pair:
    """One registration problem.

    ``target`` and ``source`` are (N, 4) float32 arrays.  ``T_gt`` is the 4x4
    float64 rigid transform that maps source coordinates onto the target, so
    a perfect registration returns a pose equal to ``T_gt``.
    """

    name: str
    target: np.ndarray
    source: np.ndarray
    T_gt: np.ndarray
    voxel_size: float = 0.0      # > 0: fixed voxel edge in metres
    grid_divisions: int = 0      # > 0: voxel edge = bounding-box extent / divisions
    iters: int = 30
    meta: dict = field(default_factory=dict)


def _as_xyzw(p: np.ndarray) -> np.ndarray:
    out = np.zeros((p.shape[0], 4), dtype=np.float32)
    out[:, :3] = p.astype(np.float32)
    return out


def _unit_vectors(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _axis_angle_matrix(axis: np.ndarray, angle: float) -> np.ndarray:
    """Rotation about a unit axis (Rodrigues' formula), float64."""
    a = axis / np.linalg.norm(axis)
    K = np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])
    return np.eye(3) + math.sin(angle) * K + (1.0 - math.cos(angle)) * (K @ K)


def random_rigid(rng: np.random.Generator, max_deg: float, max_trans: float) -> np.ndarray:
    """A rigid motion: rotation by an angle U(0, max_deg) about a uniformly
    random axis, translation uniform in the ball of radius ``max_trans``."""
    axis = _unit_vectors(rng, 1)[0]
    angle = math.radians(rng.uniform(0.0, max_deg))
    direction = _unit_vectors(rng, 1)[0]
    radius = max_trans * rng.uniform() ** (1.0 / 3.0)
    T = np.eye(4)
    T[:3, :3] = _axis_angle_matrix(axis, angle)
    T[:3, 3] = radius * direction
    return T


def _move(T: np.ndarray, p: np.ndarray) -> np.ndarray:
    return p @ T[:3, :3].T + T[:3, 3]


def _object_pair(name, rng, target_xyz, max_deg, max_trans, sigma, **kw) -> Pair:
    """Source = motion^-1 applied to the target, plus iid Gaussian noise, so
    that the pose mapping source onto target is ``T_gt``."""
    M = random_rigid(rng, max_deg, max_trans)
    src = _move(M, target_xyz) + rng.normal(0.0, sigma, size=target_xyz.shape)
    T_gt = np.linalg.inv(M)
    return Pair(name, _as_xyzw(target_xyz), _as_xyzw(src), T_gt, **kw)


# ---------------------------------------------------------------------------
# 4,096-point sphere + plane (ModelNet-sized stand-in)
# ---------------------------------------------------------------------------
def sphere_plane(seed: int = CONFIG_SEEDS[1], n: int = 4096, max_deg: float = 10.0,
                 max_trans: float = 0.05, sigma: float = 0.001) -> Pair:
    """Half the points uniform on the unit sphere, half uniform on the 1x1
    plane z = -1 (x, y in [-0.5, 0.5]); voxel edge = extent / 64."""
    rng = np.random.default_rng(seed)
    n_s = n // 2
    sphere = _unit_vectors(rng, n_s)
    plane = np.column_stack([rng.uniform(-0.5, 0.5, n - n_s), rng.uniform(-0.5, 0.5, n - n_s),
                             np.full(n - n_s, -1.0)])
    tgt = np.concatenate([sphere, plane])
    return _object_pair("sphere_plane_4k", rng, tgt, max_deg, max_trans, sigma,
                        grid_divisions=64, iters=30)


# ---------------------------------------------------------------------------
# 40,000-point bumpy closed surface (Bunny-sized stand-in)
# ---------------------------------------------------------------------------
def _real_sph_harm(lmax: int, ct: np.ndarray, phi: np.ndarray) -> list[np.ndarray]:
    """Orthonormal real spherical harmonics Y_lm, l <= lmax, evaluated at
    cos(theta) = ct and azimuth phi (associated-Legendre recurrence)."""
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    out = []
    P = {}
    for m in range(lmax + 1):
        # P_m^m, then upward in l.
        pmm = np.ones_like(ct)
        for k in range(1, m + 1):
            pmm = -pmm * (2 * k - 1) * st
        P[(m, m)] = pmm
        if m + 1 <= lmax:
            P[(m + 1, m)] = ct * (2 * m + 1) * pmm
        for l in range(m + 2, lmax + 1):
            P[(l, m)] = ((2 * l - 1) * ct * P[(l - 1, m)] - (l + m - 1) * P[(l - 2, m)]) / (l - m)
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
            if m == 0:
                out.append(norm * P[(l, 0)])
            elif m > 0:
                out.append(math.sqrt(2.0) * norm * P[(l, am)] * np.cos(am * phi))
            else:
                out.append(math.sqrt(2.0) * norm * P[(l, am)] * np.sin(am * phi))
    return out


def bumpy_object(seed: int = CONFIG_SEEDS[2], n: int = 40_000, lmax: int = 8,
                 amplitude: float = 0.1, density_ratio: float = 10.0, max_deg: float = 15.0,
                 max_trans: float = 0.1, sigma: float = 0.002) -> Pair:
    """Unit sphere radially perturbed by random real spherical harmonics up to
    degree ``lmax`` (N(0,1) coefficients, rescaled so the largest deviation is
    ``amplitude``).  Points are kept by rejection with acceptance rising
    linearly from 1/density_ratio at the south pole to 1 at the north pole."""
    rng = np.random.default_rng(seed)
    coeff = rng.standard_normal((lmax + 1) ** 2)

    def radial(dirs):
        ct = dirs[:, 2]
        phi = np.arctan2(dirs[:, 1], dirs[:, 0])
        Y = _real_sph_harm(lmax, ct, phi)
        return sum(c * y for c, y in zip(coeff, Y))

    # Scale from a dense probe of the sphere so max |deviation| = amplitude.
    probe = _unit_vectors(rng, 200_000)
    scale = amplitude / np.max(np.abs(radial(probe)))
    lo = 1.0 / density_ratio
    kept = []
    total = 0
    while total < n:
        d = _unit_vectors(rng, 2 * n)
        accept = lo + (1.0 - lo) * (1.0 + d[:, 2]) / 2.0
        d = d[rng.uniform(size=d.shape[0]) < accept]
        kept.append(d)
        total += d.shape[0]
    d = np.concatenate(kept)[:n]
    pts = d * (1.0 + scale * radial(d))[:, None]
    return _object_pair("bumpy_object_40k", rng, pts, max_deg, max_trans, sigma,
                        grid_divisions=128, iters=50)


# ---------------------------------------------------------------------------
# ~226,000-point RGB-D-like scene (TUM-sized stand-in)
# ---------------------------------------------------------------------------
_FX = _FY = 525.0
_CX, _CY = 319.5, 239.5
_W, _H = 640, 480


def _scene_objects(rng: np.random.Generator) -> list[dict]:
    """A room-like set of planes and boxes in the first camera's frame
    (x right, y down, z forward)."""
    objs = []
    # Back wall (slightly tilted), floor and one side wall: infinite planes.
    n_back = np.array([rng.uniform(-0.08, 0.08), rng.uniform(-0.05, 0.05), -1.0])
    objs.append(dict(kind="plane", n=n_back / np.linalg.norm(n_back), p=np.array([0.0, 0.0, 4.85])))
    objs.append(dict(kind="plane", n=np.array([0.0, -1.0, 0.0]), p=np.array([0.0, 1.25, 0.0])))
    objs.append(dict(kind="plane", n=np.array([1.0, 0.0, rng.uniform(-0.1, 0.1)]),
                     p=np.array([-2.7, 0.0, 0.0])))
    # Boxes resting on the floor, some rotated about the vertical axis.
    for k in range(9):
        size = rng.uniform(0.25, 1.1, 3)
        cz = rng.uniform(1.2, 4.3)
        cx = rng.uniform(-2.2, 2.4)
        center = np.array([cx, 1.25 - size[1] / 2.0, cz])
        yaw = rng.uniform(0.0, math.pi / 2.0) if k % 2 else 0.0
        objs.append(dict(kind="box", c=center, half=size / 2.0,
                         R=_axis_angle_matrix(np.array([0.0, 1.0, 0.0]), yaw)))
    # Two free-standing thin panels: one close to the optical axis at about
    # 0.6 m (so depths reach down to 0.5 m), one in the middle of the room.
    for cx, cy, z, hs in ((rng.uniform(-0.25, 0.25), rng.uniform(-0.15, 0.15), rng.uniform(0.55, 0.7), 0.12),
                          (rng.uniform(-1.0, 1.0), rng.uniform(-0.6, 0.3), rng.uniform(2.0, 3.0), 0.4)):
        tilt = _axis_angle_matrix(_unit_vectors(rng, 1)[0], math.radians(rng.uniform(10, 40)))
        objs.append(dict(kind="box", c=np.array([cx, cy, z]),
                         half=np.array([hs, 0.8 * hs, 0.01]), R=tilt))
    return objs


def _render_depth(objs, R_cam: np.ndarray, t_cam: np.ndarray) -> np.ndarray:
    """Ray-cast a 640x480 pinhole camera whose pose in the scene frame is
    (R_cam, t_cam).  Returns the z-depth image in the camera frame (inf where
    nothing is hit)."""
    u, v = np.meshgrid(np.arange(_W, dtype=np.float64), np.arange(_H, dtype=np.float64))
    d_cam = np.stack([(u - _CX) / _FX, (v - _CY) / _FY, np.ones_like(u)], axis=-1).reshape(-1, 3)
    d = d_cam @ R_cam.T                    # ray directions in the scene frame (z_cam = 1 scaling)
    o = t_cam
    best = np.full(d.shape[0], np.inf)
    with np.errstate(divide="ignore", invalid="ignore"):
        for ob in objs:
            if ob["kind"] == "plane":
                den = d @ ob["n"]
                s = ((ob["p"] - o) @ ob["n"]) / den
                s = np.where((s > 1e-6) & np.isfinite(s), s, np.inf)
            else:
                # Slab test in the box's own frame.
                Rb = ob["R"]
                ol = (o - ob["c"]) @ Rb
                dl = d @ Rb
                t1 = (-ob["half"] - ol) / dl
                t2 = (ob["half"] - ol) / dl
                tmin = np.nanmax(np.minimum(t1, t2), axis=1)
                tmax = np.nanmin(np.maximum(t1, t2), axis=1)
                hit = (tmax >= tmin) & (tmax > 1e-6)
                s = np.where(hit, np.where(tmin > 1e-6, tmin, tmax), np.inf)
            best = np.minimum(best, s)
    # Ray parameter s is the camera-frame depth because d_cam.z == 1.
    return best.reshape(_H, _W)


def _sample_depth_points(rng, depth, n_keep, zmin, zmax, invalid_frac, noise_coeff) -> np.ndarray:
    """Back-project ``n_keep`` pixels chosen without replacement with weight
    proportional to 1/z^2 (density falls with depth squared)."""
    z = depth.reshape(-1)
    valid = np.isfinite(z) & (z >= zmin) & (z <= zmax)
    valid &= rng.uniform(size=z.shape[0]) >= invalid_frac
    idx = np.flatnonzero(valid)
    if idx.shape[0] < n_keep:
        raise ValueError(f"scene has only {idx.shape[0]} valid pixels, need {n_keep}")
    w = 1.0 / (z[idx] ** 2)
    # Weighted sampling without replacement (Efraimidis-Spirakis keys).
    keys = np.log(rng.uniform(size=idx.shape[0])) / w
    pick = idx[np.argpartition(-keys, n_keep - 1)[:n_keep]]
    pick.sort()
    zz = z[pick]
    if noise_coeff > 0.0:
        zz = zz + rng.normal(0.0, 1.0, size=zz.shape[0]) * noise_coeff * zz * zz
    u = (pick % _W).astype(np.float64)
    v = (pick // _W).astype(np.float64)
    return np.column_stack([(u - _CX) * zz / _FX, (v - _CY) * zz / _FY, zz])


def depth_scene(seed: int = CONFIG_SEEDS[3], n: int = 226_000, max_deg: float = 5.0,
                max_trans: float = 0.1, voxel_size: float = 0.02) -> Pair:
    """Target: the scene seen by camera 1 (depth clipped to [0.5, 5] m, 2% of
    pixels invalid, n pixels kept with density falling as 1/z^2).  Source: the
    same scene from camera 2, moved by a rigid motion of at most ``max_deg``
    and ``max_trans``, with depth noise sigma = 0.002 z^2 and independent
    pixel sampling.  T_gt is camera 2's pose in camera 1's frame."""
    rng = np.random.default_rng(seed)
    objs = _scene_objects(rng)
    T_c = random_rigid(rng, max_deg, max_trans)
    tgt = _sample_depth_points(rng, _render_depth(objs, np.eye(3), np.zeros(3)), n,
                               0.5, 5.0, 0.02, 0.0)
    src = _sample_depth_points(rng, _render_depth(objs, T_c[:3, :3], T_c[:3, 3]), n,
                               0.5, 5.0, 0.02, 0.002)
    return Pair("depth_scene_226k", _as_xyzw(tgt), _as_xyzw(src), T_c,
                voxel_size=voxel_size, iters=30)


# ---------------------------------------------------------------------------
# Many uneven pairs
# ---------------------------------------------------------------------------
def batched_pairs(seed: int = CONFIG_SEEDS[4], n_pairs: int = 256, n_min: int = 2000,
                  n_max: int = 64000) -> list[Pair]:
    """Pairs with sizes log-uniform in [n_min, n_max]; even pairs use the
    sphere+plane generator, odd pairs the bumpy-object generator; motions of
    at most 15 degrees and 0.1 x extent."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_pairs):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        sub = int(rng.integers(0, 2**31 - 1))
        if k % 2 == 0:
            p = sphere_plane(seed=sub, n=n, max_deg=15.0, max_trans=0.2, sigma=0.001)
        else:
            p = bumpy_object(seed=sub, n=n, max_deg=15.0, max_trans=0.2, sigma=0.002)
        p.name = f"pair{k:03d}_{p.name.split('_')[0]}_{n}"
        p.iters = 40
        out.append(p)
    return out


def _loss_pair(args):
    k, seed, n = args
    p = bumpy_object(seed=seed, n=n)
    p.name = f"loss{k:02d}_{n}"
    return p


def loss_pairs(seed: int = CONFIG_SEEDS[5], n_pairs: int = 64, n: int = 20_000, workers: int = 1) -> list[Pair]:
    """The differentiable-loss workload: pairs of n points from the
    bumpy-object generator (voxel = extent / 128).  Each pair's seed is drawn
    first, so `workers` > 1 (processes, started by spawning) gives the same
    pairs."""
    rng = np.random.default_rng(seed)
    jobs = [(k, int(rng.integers(0, 2**31 - 1)), n) for k in range(n_pairs)]
    if workers <= 1:
        return [_loss_pair(j) for j in jobs]
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_loss_pair, jobs))


def make_config(k: int) -> Pair:
    """The single-pair workloads by number: 1 sphere+plane 4k, 2 bumpy object
    40k, 3 depth scene 226k."""
    if k == 1:
        return sphere_plane()
    if k == 2:
        return bumpy_object()
    if k == 3:
        return depth_scene()
    raise ValueError(f"no single-pair workload {k}")
