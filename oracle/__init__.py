"""CPU oracle for the dilation-based ICP hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  It wraps ``vicp_oracle.c``, a
plain C restatement of the paper's steps (Alg. 1-4, Eq. 1), through ctypes.
It imports nothing from the CUDA package and the CUDA package imports nothing
from it.

The C file is built twice: single-threaded (the default), and with OpenMP
over the loops whose iterations are independent (keys, one dilation round,
the searches); ``use_threads(n)`` selects the second for n > 1.  Both give
bit-identical results (pinned in ``tests/test_oracle_threads.py``).

Functions take and return numpy arrays.  Point clouds are (N, 4) float32,
C-contiguous (x, y, z, w; w ignored).  Poses are 4x4 float64 row-major.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vicp_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libvicp_oracle.so")
_LIB_OMP = os.path.join(_LIB_DIR, "libvicp_oracle_omp.so")
_lock = threading.Lock()
_libs = {}          # "plain" / "omp" -> CDLL
_threads = 1        # threads of the calls that follow (1: the plain build)

OK = 0
ERR_INVALID = 1
ERR_DEGENERATE = 7


def _compile(lib: str, extra, force: bool) -> bool:
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(_SRC):
        return True
    tmp = lib + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", *extra,
           "-o", tmp, _SRC, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        return False
    os.replace(tmp, lib)
    return True


def build(force: bool = False) -> str:
    """Compile the oracle with gcc, single-threaded and (where gcc has
    OpenMP) multi-threaded.  -ffp-contract=off keeps every float operation
    separately rounded (gcc contracts a*b+c into FMA by default on aarch64),
    which the bit-exact comparisons rely on."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if not _compile(_LIB, [], force):
        raise RuntimeError("gcc failed to build the oracle")
    _compile(_LIB_OMP, ["-fopenmp"], force)   # optional: use_threads() reports 1 without it
    return _LIB


class _Grid(C.Structure):
    _fields_ = [("origin", C.c_float * 3), ("h", C.c_float), ("inv_h", C.c_float),
                ("dims", C.c_int32 * 3)]


@dataclass(frozen=True)
class Grid:
    """Voxel grid geometry: origin (float32 x3), edge h, inv_h = (float)(1/(double)h), dims."""

    origin: tuple
    h: float
    inv_h: float
    dims: tuple

    @property
    def n_voxels(self) -> int:
        return int(self.dims[0]) * int(self.dims[1]) * int(self.dims[2])

    def _c(self) -> _Grid:
        g = _Grid()
        for a in range(3):
            g.origin[a] = self.origin[a]
            g.dims[a] = self.dims[a]
        g.h = self.h
        g.inv_h = self.inv_h
        return g


def _open(which: str):
    """The CDLL of one build, loaded once ("plain" or "omp"; None if the
    OpenMP build is not available)."""
    with _lock:
        if which not in _libs:
            build()
            path = _LIB if which == "plain" else _LIB_OMP
            if not os.path.exists(path):
                _libs[which] = None
                return None
            lib = C.CDLL(path)
            P = C.c_void_p
            i32, i64, f32, f64 = C.c_int32, C.c_int64, C.c_float, C.c_double
            G = C.POINTER(_Grid)
            sig = {
                "og_fit_grid": (C.c_int, [P, i32, f32, i32, G]),
                "og_num_voxels": (i64, [G]),
                "og_voxel_key": (i32, [G, f32, f32, f32]),
                "og_keys": (None, [G, P, i32, P]),
                "og_histogram": (None, [P, i32, i64, P]),
                "og_offsets": (None, [P, i64, P]),
                "og_paper_moc": (None, [P, i64, P]),
                "og_paper_static_bytes": (i64, [i64]),
                "og_csr": (None, [P, i32, P, i64, P]),
                "og_dilate": (None, [G, P, i32, P, P]),
                "og_correspond": (None, [G, P, P, P, P, i32, P, i32, P, P, P, P]),
                "og_reduce": (None, [P, P, i32, P, P, P, P, P, P]),
                "og_svd3": (None, [P, P, P, P]),
                "og_is_degenerate": (C.c_int, [P]),
                "og_solve": (C.c_int, [P, P, P, P]),
                "og_compose": (None, [P, P]),
                "og_build": (None, [G, P, i32, i32, P, P, P, P, P, P]),
                "og_iterate": (C.c_int, [G, P, P, P, P, i32, P, i32, P, P, P, P, P, P]),
                "og_register": (C.c_int, [G, i32, P, i32, P, i32, P, i32, f64, P, P]),
                "og_set_threads": (i32, [i32]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _libs[which] = lib
    return _libs[which]


def _load():
    if _threads > 1:
        lib = _open("omp")
        if lib is not None:
            return lib
    return _open("plain")


def use_threads(n: int) -> int:
    """Run the following calls on n threads (n <= 1: the single-threaded
    build).  Returns the thread count the calls will use (1 where gcc has no
    OpenMP)."""
    global _threads
    n = int(n)
    if n <= 1:
        _threads = 1
        return 1
    lib = _open("omp")
    if lib is None:
        _threads = 1
        return 1
    _threads = int(lib.og_set_threads(n))
    return _threads


def threads() -> int:
    """Threads the oracle's calls use now."""
    return _threads


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _pts(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] != 4:
        raise ValueError("point clouds are (N, 4) float32")
    return a


def _pose(T) -> np.ndarray:
    T = np.ascontiguousarray(T, dtype=np.float64)
    if T.shape != (4, 4):
        raise ValueError("pose is 4x4 float64")
    return T


# ---------------------------------------------------------------------------
# Geometry
# ---------------------------------------------------------------------------
def fit_grid(target, voxel_size: float = 0.0, divisions: int = 0) -> Grid:
    """Bounding-box grid over the target (origin = min corner)."""
    t = _pts(target)
    g = _Grid()
    st = _load().og_fit_grid(_ptr(t), t.shape[0], float(voxel_size), int(divisions), C.byref(g))
    if st != OK:
        raise ValueError(f"og_fit_grid failed with status {st}")
    return Grid(tuple(float(np.float32(g.origin[a])) for a in range(3)), float(np.float32(g.h)),
                float(np.float32(g.inv_h)), tuple(int(g.dims[a]) for a in range(3)))


def explicit_grid(origin, h: float, dims) -> Grid:
    """A grid with caller-chosen origin, edge and dims."""
    h32 = float(np.float32(h))
    inv_h = float(np.float32(1.0 / h32))
    return Grid(tuple(float(np.float32(o)) for o in origin), h32, inv_h, tuple(int(d) for d in dims))


def voxel_key(grid: Grid, x: float, y: float, z: float) -> int:
    g = grid._c()
    return int(_load().og_voxel_key(C.byref(g), x, y, z))


# ---------------------------------------------------------------------------
# Grid build steps (Alg. 1-3)
# ---------------------------------------------------------------------------
def keys(grid: Grid, pts) -> np.ndarray:
    p = _pts(pts)
    out = np.empty(p.shape[0], dtype=np.int32)
    g = grid._c()
    _load().og_keys(C.byref(g), _ptr(p), p.shape[0], _ptr(out))
    return out


def histogram(keys_: np.ndarray, n_voxels: int) -> np.ndarray:
    k = np.ascontiguousarray(keys_, dtype=np.int32)
    out = np.empty(n_voxels, dtype=np.uint32)
    _load().og_histogram(_ptr(k), k.shape[0], n_voxels, _ptr(out))
    return out


def offsets(counts: np.ndarray) -> np.ndarray:
    c = np.ascontiguousarray(counts, dtype=np.uint32)
    out = np.empty(c.shape[0] + 1, dtype=np.uint32)
    _load().og_offsets(_ptr(c), c.shape[0], _ptr(out))
    return out


def paper_moc(counts: np.ndarray) -> np.ndarray:
    c = np.ascontiguousarray(counts, dtype=np.uint32)
    out = np.empty(c.shape[0], dtype=np.uint32)
    _load().og_paper_moc(_ptr(c), c.shape[0], _ptr(out))
    return out


def paper_static_bytes(n_voxels: int) -> int:
    return int(_load().og_paper_static_bytes(n_voxels))


def csr(keys_: np.ndarray, off: np.ndarray) -> np.ndarray:
    k = np.ascontiguousarray(keys_, dtype=np.int32)
    o = np.ascontiguousarray(off, dtype=np.uint32)
    out = np.empty(int(o[-1]), dtype=np.int32)
    _load().og_csr(_ptr(k), k.shape[0], _ptr(o), o.shape[0] - 1, _ptr(out))
    return out


def dilate(grid: Grid, off: np.ndarray, layers: int):
    o = np.ascontiguousarray(off, dtype=np.uint32)
    V = grid.n_voxels
    if o.shape[0] != V + 1:
        raise ValueError("offsets must have V+1 entries")
    if not 0 <= layers <= 254:
        raise ValueError("oracle dilation supports 0 <= L <= 254")
    root = np.empty(V, dtype=np.int32)
    ring = np.empty(V, dtype=np.uint8)
    g = grid._c()
    _load().og_dilate(C.byref(g), _ptr(o), int(layers), _ptr(root), _ptr(ring))
    return root, ring


def build_grid(grid: Grid, target, layers: int) -> dict:
    """Keys, counts, offsets, CSR ids, root and ring for one target cloud."""
    t = _pts(target)
    n, V = t.shape[0], grid.n_voxels
    out = dict(keys=np.empty(n, np.int32), counts=np.empty(V, np.uint32),
               off=np.empty(V + 1, np.uint32), ids=np.empty(n, np.int32),
               root=np.empty(V, np.int32), ring=np.empty(V, np.uint8))
    g = grid._c()
    _load().og_build(C.byref(g), _ptr(t), n, int(layers), _ptr(out["keys"]), _ptr(out["counts"]),
                     _ptr(out["off"]), _ptr(out["ids"]), _ptr(out["root"]), _ptr(out["ring"]))
    out["ids"] = out["ids"][: int(out["off"][-1])]
    return out


# ---------------------------------------------------------------------------
# NNS, reduction and solve (Alg. 4, Eq. 1)
# ---------------------------------------------------------------------------
def correspond(grid: Grid, built: dict, target, source, pose):
    """Returns (nn int32[M], d2 float32[M], fallback bool[M])."""
    t, s, T = _pts(target), _pts(source), _pose(pose)
    m = s.shape[0]
    nn = np.empty(m, np.int32)
    d2 = np.empty(m, np.float32)
    fb = np.empty(m, np.uint8)
    ids = np.ascontiguousarray(built["ids"], dtype=np.int32)
    if ids.shape[0] == 0:
        ids = np.zeros(1, np.int32)
    g = grid._c()
    _load().og_correspond(C.byref(g), _ptr(built["off"]), _ptr(ids), _ptr(built["root"]), _ptr(t),
                          t.shape[0], _ptr(s), m, _ptr(T), _ptr(nn), _ptr(d2), _ptr(fb))
    return nn, d2, fb.astype(bool)


def reduce(target, source, pose, nn):
    """Returns (pbar[3], qbar[3], H 3x3, rmse) in float64."""
    t, s, T = _pts(target), _pts(source), _pose(pose)
    nn_ = np.ascontiguousarray(nn, dtype=np.int32)
    pbar, qbar, H, rmse = np.empty(3), np.empty(3), np.empty(9), np.empty(1)
    _load().og_reduce(_ptr(t), _ptr(s), s.shape[0], _ptr(T), _ptr(nn_), _ptr(pbar), _ptr(qbar),
                      _ptr(H), _ptr(rmse))
    return pbar, qbar, H.reshape(3, 3), float(rmse[0])


def svd3(H):
    """H = U diag(sig) V^T by the oracle's one-sided Jacobi."""
    Hc = np.ascontiguousarray(H, dtype=np.float64).reshape(9)
    U, sig, V = np.empty(9), np.empty(3), np.empty(9)
    _load().og_svd3(_ptr(Hc), _ptr(U), _ptr(sig), _ptr(V))
    return U.reshape(3, 3), sig, V.reshape(3, 3)


def is_degenerate(H) -> bool:
    Hc = np.ascontiguousarray(H, dtype=np.float64).reshape(9)
    return bool(_load().og_is_degenerate(_ptr(Hc)))


def solve(pbar, qbar, H):
    """Returns (status, dT 4x4)."""
    p = np.ascontiguousarray(pbar, dtype=np.float64)
    q = np.ascontiguousarray(qbar, dtype=np.float64)
    Hc = np.ascontiguousarray(H, dtype=np.float64).reshape(9)
    dT = np.zeros(16)
    st = _load().og_solve(_ptr(p), _ptr(q), _ptr(Hc), _ptr(dT))
    return int(st), dT.reshape(4, 4)


def compose(dT, T) -> np.ndarray:
    d = _pose(dT)
    out = _pose(T).copy()
    _load().og_compose(_ptr(d), _ptr(out))
    return out


def iterate(grid: Grid, built: dict, target, source, pose):
    """One ICP iteration.  Returns (status, new_pose, rmse, nn, d2, fallback, n_fallback)."""
    t, s = _pts(target), _pts(source)
    T = _pose(pose).copy()
    m = s.shape[0]
    nn, d2, fb = np.empty(m, np.int32), np.empty(m, np.float32), np.empty(m, np.uint8)
    rmse = np.empty(1)
    nf = C.c_int32(0)
    ids = np.ascontiguousarray(built["ids"], dtype=np.int32)
    if ids.shape[0] == 0:
        ids = np.zeros(1, np.int32)
    g = grid._c()
    st = _load().og_iterate(C.byref(g), _ptr(built["off"]), _ptr(ids), _ptr(built["root"]), _ptr(t),
                            t.shape[0], _ptr(s), m, _ptr(T), _ptr(nn), _ptr(d2), _ptr(fb),
                            _ptr(rmse), C.byref(nf))
    return int(st), T, float(rmse[0]), nn, d2, fb.astype(bool), int(nf.value)


def register(grid: Grid, layers: int, target, source, pose=None, max_iters: int = 50,
             eps: float = 1e-5):
    """Full ICP.  Returns (status, pose, iters, rmse_history)."""
    t, s = _pts(target), _pts(source)
    T = _pose(np.eye(4) if pose is None else pose).copy()
    hist = np.zeros(max(1, max_iters))
    it = C.c_int32(0)
    g = grid._c()
    st = _load().og_register(C.byref(g), int(layers), _ptr(t), t.shape[0], _ptr(s), s.shape[0],
                             _ptr(T), int(max_iters), float(eps), C.byref(it), _ptr(hist))
    return int(st), T, int(it.value), hist[: max(int(it.value), 0)]
