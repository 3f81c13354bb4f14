"""Python binding of the C ABI in ``include/vicp.h`` -- argument marshalling only.

Every step of the registration runs in the CUDA kernels of ``libvicp.so``;
this module checks tensor shapes, dtypes and devices, passes raw pointers and
the current torch CUDA stream, and turns status codes into exceptions.  The
functions carry the C names (``vicp_create``, ``vicp_build_grid``, ...); the
``Context`` class bundles them.

Point clouds are CUDA float32 tensors of shape (N, 4) (x, y, z, w; w is
ignored), contiguous and 16-byte aligned.  Poses are 4x4 float64.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np
import torch

from . import build as _build

VICP_OK = 0
VICP_ERR_INVALID = 1
VICP_ERR_CUDA = 2
VICP_ERR_OOM = 3
VICP_ERR_GRID_TOO_LARGE = 4
VICP_ERR_TIMEOUT = 5
VICP_ERR_STATE = 6
VICP_ERR_DEGENERATE = 7

VICP_STATIC_MAX_VOXELS = 1 << 24
VICP_STATIC_MAX_BRICK_SLOTS = 1 << 20
VICP_FLAG_KEEP_GRID = 1 << 0
VICP_FLAG_REBUILD_EACH_ITER = 1 << 1
VICP_FLAG_FP64_SOLVE = 1 << 2
VICP_FLAG_SPARSE_GRID = 1 << 3
VICP_FLAG_NO_GRAPH = 1 << 4
VICP_HIST_WARP_AGGREGATED = 0
VICP_HIST_SHARED_HASH = 1
VICP_BATCH_MAX_PAIRS = 65536
VICP_BATCH_SHAPES = 7
VICP_BATCH_FLAG_NO_GRAPH = 1 << 0
VICP_BATCH_FLAG_TEST_BARRIER_TIMEOUT = 1 << 1
VICP_BATCH_FLAG_FP64 = 1 << 2


class VicpError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"vicp status {status}: {message}")
        self.status = status


class vicp_params(C.Structure):
    _fields_ = [("voxel_size", C.c_float), ("grid_divisions", C.c_int32), ("origin", C.c_float * 3),
                ("dims", C.c_int32 * 3), ("dilation_layers", C.c_int32), ("max_iters", C.c_int32),
                ("rmse_eps", C.c_double), ("flags", C.c_uint32)]


class vicp_grid_view(C.Structure):
    _fields_ = [("origin", C.c_float * 3), ("voxel_size", C.c_float), ("inv_voxel_size", C.c_float),
                ("dims", C.c_int32 * 3), ("n_voxels", C.c_int64), ("n_target", C.c_int32),
                ("n_stored", C.c_int32), ("dilation_layers", C.c_int32), ("keys", C.c_void_p),
                ("offsets", C.c_void_p), ("ids", C.c_void_p), ("csr_points", C.c_void_p),
                ("root", C.c_void_p), ("ring", C.c_void_p), ("occupancy", C.c_void_p)]


class vicp_memory(C.Structure):
    _fields_ = [("current_bytes", C.c_uint64), ("peak_bytes", C.c_uint64), ("static_bytes", C.c_uint64),
                ("csr_store_bytes", C.c_uint64), ("fixed_capacity_bytes", C.c_uint64),
                ("paper_static_layout_bytes", C.c_uint64), ("max_voxel_count", C.c_uint32),
                ("occupied_voxels", C.c_uint32), ("nonempty_bricks", C.c_uint32), ("labelled_voxels", C.c_uint32)]


class vicp_sparse_view(C.Structure):
    _fields_ = [("origin", C.c_float * 3), ("voxel_size", C.c_float), ("inv_voxel_size", C.c_float),
                ("dims", C.c_int32 * 3), ("n_voxels", C.c_int64), ("n_target", C.c_int32),
                ("n_stored", C.c_int32), ("dilation_layers", C.c_int32), ("occupied_slots", C.c_int64),
                ("occupied_keys", C.c_void_p), ("occupied_offsets", C.c_void_p), ("labelled_slots", C.c_int64),
                ("labelled_keys", C.c_void_p), ("labelled_segments", C.c_void_p), ("labelled_root", C.c_void_p),
                ("labelled_voxels", C.c_int64), ("labelled_segment_count", C.c_int64),
                ("keys", C.c_void_p), ("ids", C.c_void_p), ("csr_points", C.c_void_p), ("occupancy", C.c_void_p)]


class vicp_batch_params(C.Structure):
    _fields_ = [("dilation_layers", C.c_int32), ("max_iters", C.c_int32), ("rmse_eps", C.c_double),
                ("shape", C.c_int32), ("flags", C.c_uint32)]


class vicp_stats(C.Structure):
    _fields_ = [("queries", C.c_uint64), ("fallbacks", C.c_uint64), ("local_candidates", C.c_uint64),
                ("global_candidates", C.c_uint64)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class vicp_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


# Every exported symbol with its signature (also used by the ABI test).
_P = C.c_void_p
SIGNATURES = {
    "vicp_abi_version": (C.c_int32, []),
    "vicp_status_string": (C.c_char_p, [C.c_int]),
    "vicp_default_params": (None, [C.POINTER(vicp_params)]),
    "vicp_create": (C.c_int, [C.POINTER(_P), C.POINTER(vicp_params), C.POINTER(vicp_allocator), _P]),
    "vicp_destroy": (None, [_P]),
    "vicp_set_stream": (C.c_int, [_P, _P]),
    "vicp_build_grid": (C.c_int, [_P, _P, C.c_int32]),
    "vicp_dilate": (C.c_int, [_P, C.c_int32]),
    "vicp_correspond": (C.c_int, [_P, _P, C.c_int32, _P, _P, _P, _P]),
    "vicp_step": (C.c_int, [_P, _P, C.c_int32, _P, _P]),
    "vicp_register": (C.c_int, [_P, _P, C.c_int32, _P, C.c_int32, _P, C.POINTER(C.c_int32),
                                C.POINTER(C.c_double)]),
    "vicp_register_host": (C.c_int, [_P, _P, C.c_int32, _P, C.c_int32, _P, C.POINTER(C.c_int32),
                                     C.POINTER(C.c_double)]),
    "vicp_get_grid": (C.c_int, [_P, C.POINTER(vicp_grid_view)]),
    "vicp_get_sparse_grid": (C.c_int, [_P, C.POINTER(vicp_sparse_view)]),
    "vicp_sync": (C.c_int, [_P]),
    "vicp_memory_report": (C.c_int, [_P, C.POINTER(vicp_memory)]),
    "vicp_profile_enable": (C.c_int, [_P, C.c_int32]),
    "vicp_kernel_count": (C.c_int32, []),
    "vicp_kernel_name": (C.c_char_p, [C.c_int32]),
    "vicp_profile_read": (C.c_int, [_P, _P, _P]),
    "vicp_read_stats": (C.c_int, [_P, C.POINTER(vicp_stats), C.c_int32]),
    "vicp_launch_count": (C.c_int64, [_P]),
    "vicp_graph_replayed": (C.c_int32, [_P]),
    "vicp_last_error": (C.c_char_p, [_P]),
    "vicp_offsets_static": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_float), C.c_float, C.POINTER(C.c_int32), _P, _P,
                                      _P]),
    "vicp_fixed_build": (C.c_int, [_P, _P, C.c_int32, C.c_int32, C.POINTER(C.c_uint32), C.POINTER(C.c_uint64)]),
    "vicp_fixed_correspond": (C.c_int, [_P, _P, C.c_int32, _P, _P, _P, _P]),
    "vicp_fixed_view": (C.c_int, [_P, C.POINTER(_P), C.POINTER(_P), C.POINTER(C.c_int32)]),
    "vicp_voxel_histogram": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_float), C.c_float, C.POINTER(C.c_int32),
                                       C.c_int32, _P, _P, _P]),
    "vicp_batch_default_params": (None, [C.POINTER(vicp_batch_params)]),
    "vicp_batch_shape_info": (C.c_int, [C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                        C.POINTER(C.c_int32)]),
    "vicp_batch_create": (C.c_int, [C.POINTER(_P), C.POINTER(vicp_batch_params), C.POINTER(vicp_allocator), _P]),
    "vicp_batch_destroy": (None, [_P]),
    "vicp_batch_build": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P]),
    "vicp_batch_register": (C.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "vicp_batch_register_host": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "vicp_batch_correspond": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "vicp_batch_tune": (C.c_int, [_P, _P, _P, _P, C.c_int32, C.c_int32, C.POINTER(C.c_int32), _P]),
    "vicp_batch_pair_grid": (C.c_int, [_P, C.c_int32, C.POINTER(vicp_grid_view)]),
    "vicp_batch_report": (C.c_int, [_P, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.POINTER(vicp_stats),
                                    C.c_int32]),
    "vicp_batch_launch_count": (C.c_int64, [_P]),
    "vicp_batch_graph_replayed": (C.c_int32, [_P]),
    "vicp_batch_set_flags": (C.c_int, [_P, C.c_uint32]),
    "vicp_se3_exp": (C.c_int, [C.c_int32, _P, _P, _P, _P]),
    "vicp_se3_left_jacobian_t": (C.c_int, [C.c_int32, _P, _P, _P, _P]),
    "vicp_batch_loss": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "vicp_batch_last_error": (C.c_char_p, [_P]),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = False) -> C.CDLL:
    """Load libvicp.so.  Raises if it has not been built: there is no
    fallback path."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB):
                if not build_if_missing:
                    raise RuntimeError(f"{_build.LIB} is not built; run __graft_entry__.build() or "
                                       "python -m paper_2512_04996_gb300.build")
                _build.build_library()
            lib = C.CDLL(_build.LIB)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def default_params(**overrides) -> vicp_params:
    p = vicp_params()
    load_library().vicp_default_params(C.byref(p))
    for k, v in overrides.items():
        if k in ("origin", "dims"):
            arr = getattr(p, k)
            for a in range(3):
                arr[a] = v[a]
        else:
            setattr(p, k, v)
    return p


def _cloud(t: torch.Tensor, what: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32:
        raise TypeError(f"{what}: expected a CUDA float32 tensor")
    if t.dim() != 2 or t.shape[1] != 4 or not t.is_contiguous():
        raise ValueError(f"{what}: expected a contiguous (N, 4) tensor, got {tuple(t.shape)}")
    if t.data_ptr() % 16:
        raise ValueError(f"{what}: data must be 16-byte aligned")
    return t


def _host_cloud(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] != 4:
        raise ValueError("host clouds are (N, 4) float32")
    return a


class _DevArray:
    """__cuda_array_interface__ view of context-owned device memory."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"data": (ptr, False), "shape": tuple(shape), "typestr": typestr,
                                         "version": 3, "strides": None}


def _view(ptr, shape, typestr, dtype, device):
    if not ptr or 0 in shape:
        return torch.empty(shape, dtype=dtype, device=device)
    return torch.as_tensor(_DevArray(ptr, shape, typestr), device=device)


class Context:
    """One vicp context on the current CUDA device and torch stream."""

    def __init__(self, params: vicp_params | None = None, stream: torch.cuda.Stream | None = None,
                 allocator: vicp_allocator | None = None, **overrides):
        self._lib = load_library()
        self.params = params if params is not None else default_params(**overrides)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._allocator = allocator   # keep the callbacks alive
        h = C.c_void_p()
        st = self._lib.vicp_create(C.byref(h), C.byref(self.params),
                                   C.byref(allocator) if allocator is not None else None,
                                   C.c_void_p(self.stream.cuda_stream))
        if st != VICP_OK:
            raise VicpError(st, "vicp_create failed")
        self.handle = h

    # -- plumbing ---------------------------------------------------------
    def _check(self, st: int, what: str):
        if st != VICP_OK:
            raise VicpError(st, f"{what}: {self._lib.vicp_last_error(self.handle).decode()}")

    def close(self):
        if getattr(self, "handle", None):
            self._lib.vicp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- the hot path -----------------------------------------------------
    def build_grid(self, target: torch.Tensor):
        t = _cloud(target, "target")
        self._target = t   # the grid refers to it until the next build
        self._check(self._lib.vicp_build_grid(self.handle, t.data_ptr(), t.shape[0]), "vicp_build_grid")

    def dilate(self, layers: int = -1):
        self._check(self._lib.vicp_dilate(self.handle, int(layers)), "vicp_dilate")

    def correspond(self, source: torch.Tensor, pose: torch.Tensor, nn: torch.Tensor | None = None,
                   d2: torch.Tensor | None = None, n_fallback: torch.Tensor | None = None):
        s = _cloud(source, "source")
        m = s.shape[0]
        if pose.dtype != torch.float64 or not pose.is_cuda or pose.numel() != 16 or not pose.is_contiguous():
            raise ValueError("pose: contiguous CUDA float64 tensor with 16 entries")
        nn = torch.empty(m, dtype=torch.int32, device=s.device) if nn is None else nn
        d2 = torch.empty(m, dtype=torch.float32, device=s.device) if d2 is None else d2
        if n_fallback is None:
            n_fallback = torch.zeros(1, dtype=torch.int32, device=s.device)
        self._check(self._lib.vicp_correspond(self.handle, s.data_ptr(), m, pose.data_ptr(), nn.data_ptr(),
                                              d2.data_ptr(), n_fallback.data_ptr()), "vicp_correspond")
        return nn, d2, n_fallback

    def step(self, source: torch.Tensor, pose: torch.Tensor, rmse: torch.Tensor | None = None):
        s = _cloud(source, "source")
        if pose.dtype != torch.float64 or not pose.is_cuda or pose.numel() != 16 or not pose.is_contiguous():
            raise ValueError("pose: contiguous CUDA float64 tensor with 16 entries")
        rptr = 0 if rmse is None else rmse.data_ptr()
        self._check(self._lib.vicp_step(self.handle, s.data_ptr(), s.shape[0], pose.data_ptr(), rptr),
                    "vicp_step")
        return rmse

    def fixed_build(self, target: torch.Tensor, capacity: int):
        """Fixed-capacity store on the grid of the last build_grid (same
        target).  Returns (points dropped, bytes of the store)."""
        t = _cloud(target, "target")
        over, nbytes = C.c_uint32(0), C.c_uint64(0)
        self._check(self._lib.vicp_fixed_build(self.handle, t.data_ptr(), t.shape[0], int(capacity), C.byref(over),
                                               C.byref(nbytes)), "vicp_fixed_build")
        return int(over.value), int(nbytes.value)

    def fixed_correspond(self, source: torch.Tensor, pose: torch.Tensor, nn=None, d2=None, n_fallback=None):
        s = _cloud(source, "source")
        m = s.shape[0]
        if pose.dtype != torch.float64 or not pose.is_cuda or pose.numel() != 16 or not pose.is_contiguous():
            raise ValueError("pose: contiguous CUDA float64 tensor with 16 entries")
        nn = torch.empty(m, dtype=torch.int32, device=s.device) if nn is None else nn
        d2 = torch.empty(m, dtype=torch.float32, device=s.device) if d2 is None else d2
        if n_fallback is None:
            n_fallback = torch.zeros(1, dtype=torch.int32, device=s.device)
        self._check(self._lib.vicp_fixed_correspond(self.handle, s.data_ptr(), m, pose.data_ptr(), nn.data_ptr(),
                                                    d2.data_ptr(), n_fallback.data_ptr()), "vicp_fixed_correspond")
        return nn, d2, n_fallback

    def fixed_view(self) -> dict:
        """Copies of the fixed-capacity store: slots (V * C, 4) float32 and
        fill counts (V,) int32 holding uint32, with the capacity C."""
        slots, fill, cap = C.c_void_p(), C.c_void_p(), C.c_int32(0)
        self._check(self._lib.vicp_fixed_view(self.handle, C.byref(slots), C.byref(fill), C.byref(cap)),
                    "vicp_fixed_view")
        V = int(self.grid_view().n_voxels)
        Cap = int(cap.value)
        return {"capacity": Cap,
                "slots": _view(slots.value, (V * Cap, 4), "<f4", torch.float32, self.device).clone(),
                "fill": _view(fill.value, (V,), "<u4", torch.uint32, self.device).clone()}

    def register(self, source: torch.Tensor, target: torch.Tensor, pose=None):
        s, t = _cloud(source, "source"), _cloud(target, "target")
        self._target = t
        P = np.ascontiguousarray(np.eye(4) if pose is None else pose, dtype=np.float64).copy()
        it, rm = C.c_int32(0), C.c_double(0.0)
        st = self._lib.vicp_register(self.handle, s.data_ptr(), s.shape[0], t.data_ptr(), t.shape[0],
                                     P.ctypes.data_as(C.c_void_p), C.byref(it), C.byref(rm))
        return st, P, int(it.value), float(rm.value)

    def register_host(self, source, target, pose=None):
        s, t = _host_cloud(source), _host_cloud(target)
        P = np.ascontiguousarray(np.eye(4) if pose is None else pose, dtype=np.float64).copy()
        it, rm = C.c_int32(0), C.c_double(0.0)
        st = self._lib.vicp_register_host(self.handle, s.ctypes.data_as(C.c_void_p), s.shape[0],
                                          t.ctypes.data_as(C.c_void_p), t.shape[0],
                                          P.ctypes.data_as(C.c_void_p), C.byref(it), C.byref(rm))
        return st, P, int(it.value), float(rm.value)

    # -- inspection -------------------------------------------------------
    def sync(self) -> int:
        return int(self._lib.vicp_sync(self.handle))

    def last_error(self) -> str:
        return self._lib.vicp_last_error(self.handle).decode()

    def grid_view(self) -> vicp_grid_view:
        v = vicp_grid_view()
        self._check(self._lib.vicp_get_grid(self.handle, C.byref(v)), "vicp_get_grid")
        return v

    def get_grid(self) -> dict:
        """Copies of the grid arrays as torch tensors on the device."""
        v = self.grid_view()
        V, n, ns = int(v.n_voxels), int(v.n_target), int(v.n_stored)
        d = self.device
        out = {
            "origin": tuple(float(v.origin[a]) for a in range(3)), "voxel_size": float(v.voxel_size),
            "inv_voxel_size": float(v.inv_voxel_size), "dims": tuple(int(v.dims[a]) for a in range(3)),
            "n_voxels": V, "n_target": n, "n_stored": ns, "dilation_layers": int(v.dilation_layers),
            "keys": _view(v.keys, (n,), "<i4", torch.int32, d).clone(),
            "offsets": _view(v.offsets, (V + 1,), "<u4", torch.uint32, d).clone(),
            "ids": _view(v.ids, (ns,), "<i4", torch.int32, d).clone(),
            "csr_points": _view(v.csr_points, (ns, 4), "<f4", torch.float32, d).clone(),
            "occupancy": _view(v.occupancy, ((V + 31) // 32,), "<u4", torch.uint32, d).clone(),
        }
        if v.dilation_layers >= 0:
            out["root"] = _view(v.root, (V,), "<i4", torch.int32, d).clone()
            out["ring"] = _view(v.ring, (V,), "|u1", torch.uint8, d).clone()
        return out

    def get_sparse_grid(self) -> dict:
        """Copies of the sparse grid's arrays (a context created with
        VICP_FLAG_SPARSE_GRID) as torch tensors on the device."""
        v = vicp_sparse_view()
        self._check(self._lib.vicp_get_sparse_grid(self.handle, C.byref(v)), "vicp_get_sparse_grid")
        V, n, ns = int(v.n_voxels), int(v.n_target), int(v.n_stored)
        So, Sl = int(v.occupied_slots), int(v.labelled_slots)
        d = self.device
        return {
            "origin": tuple(float(v.origin[a]) for a in range(3)), "voxel_size": float(v.voxel_size),
            "inv_voxel_size": float(v.inv_voxel_size), "dims": tuple(int(v.dims[a]) for a in range(3)),
            "n_voxels": V, "n_target": n, "n_stored": ns, "dilation_layers": int(v.dilation_layers),
            "labelled_voxels": int(v.labelled_voxels), "labelled_segment_count": int(v.labelled_segment_count),
            "occupied_keys": _view(v.occupied_keys, (So,), "<u4", torch.uint32, d).clone(),
            "occupied_offsets": _view(v.occupied_offsets, (So + 1,), "<u4", torch.uint32, d).clone(),
            "labelled_keys": _view(v.labelled_keys, (Sl,), "<u4", torch.uint32, d).clone(),
            "labelled_segments": _view(v.labelled_segments, (Sl, 2), "<u4", torch.uint32, d).clone(),
            "labelled_root": _view(v.labelled_root, (int(v.labelled_voxels),), "<i4", torch.int32, d).clone(),
            "keys": _view(v.keys, (n,), "<i4", torch.int32, d).clone(),
            "ids": _view(v.ids, (ns,), "<i4", torch.int32, d).clone(),
            "csr_points": _view(v.csr_points, (ns, 4), "<f4", torch.float32, d).clone(),
            "occupancy": _view(v.occupancy, ((V + 31) // 32,), "<u4", torch.uint32, d).clone(),
        }

    def memory_report(self) -> dict:
        m = vicp_memory()
        self._check(self._lib.vicp_memory_report(self.handle, C.byref(m)), "vicp_memory_report")
        return {name: int(getattr(m, name)) for name, _ in vicp_memory._fields_}

    def profile_enable(self, on: bool = True):
        self._check(self._lib.vicp_profile_enable(self.handle, 1 if on else 0), "vicp_profile_enable")

    def profile_read(self) -> dict:
        k = int(self._lib.vicp_kernel_count())
        launches = np.zeros(k, np.int64)
        ms = np.zeros(k, np.float64)
        self._check(self._lib.vicp_profile_read(self.handle, launches.ctypes.data_as(C.c_void_p),
                                                ms.ctypes.data_as(C.c_void_p)), "vicp_profile_read")
        return {self._lib.vicp_kernel_name(i).decode(): (int(launches[i]), float(ms[i])) for i in range(k)}

    def read_stats(self, reset: bool = True) -> dict:
        st = vicp_stats()
        self._check(self._lib.vicp_read_stats(self.handle, C.byref(st), 1 if reset else 0), "vicp_read_stats")
        return {name: int(getattr(st, name)) for name, _ in vicp_stats._fields_}

    def launch_count(self) -> int:
        return int(self._lib.vicp_launch_count(self.handle))

    def graph_replayed(self) -> bool:
        """Whether the last register / register_host call replayed its
        captured CUDA graph."""
        return bool(self._lib.vicp_graph_replayed(self.handle))


# --- the C names, as plain functions over a Context ------------------------
def vicp_create(params: vicp_params | None = None, stream=None, allocator=None, **overrides) -> Context:
    return Context(params, stream, allocator, **overrides)


def vicp_destroy(ctx: Context):
    ctx.close()


def vicp_build_grid(ctx: Context, target):
    ctx.build_grid(target)


def vicp_dilate(ctx: Context, layers: int = -1):
    ctx.dilate(layers)


def vicp_correspond(ctx: Context, source, pose, nn=None, d2=None, n_fallback=None):
    return ctx.correspond(source, pose, nn, d2, n_fallback)


def vicp_step(ctx: Context, source, pose, rmse=None):
    return ctx.step(source, pose, rmse)


def vicp_register(ctx: Context, source, target, pose=None):
    return ctx.register(source, target, pose)


def vicp_register_host(ctx: Context, source, target, pose=None):
    return ctx.register_host(source, target, pose)


def vicp_get_grid(ctx: Context) -> dict:
    return ctx.get_grid()


def vicp_sync(ctx: Context) -> int:
    return ctx.sync()


def vicp_memory_report(ctx: Context) -> dict:
    return ctx.memory_report()


def vicp_offsets_static(target, origin, voxel_size: float, dims, keys=None, offsets=None, stream=None):
    """Voxel keys and segment offsets of `target` on an explicit grid, computed
    in the library's static scratch without any device allocation by the
    library (the output tensors below are allocated here only when not
    given).  Returns (keys int32[n], offsets int32[V + 1] holding uint32
    values).  Calls must not overlap in time on one device."""
    lib = load_library()
    _cloud(target, "target")
    n = target.shape[0]
    V = int(dims[0]) * int(dims[1]) * int(dims[2])
    if V > VICP_STATIC_MAX_VOXELS:   # before sizing any output
        raise VicpError(VICP_ERR_GRID_TOO_LARGE, f"vicp_offsets_static: {V} voxels, the static scratch holds "
                                                 f"at most {VICP_STATIC_MAX_VOXELS}")
    if keys is None:
        keys = torch.empty(n, dtype=torch.int32, device=target.device)
    if offsets is None:
        offsets = torch.empty(V + 1, dtype=torch.int32, device=target.device)
    for t, size, what in ((keys, n, "keys"), (offsets, V + 1, "offsets")):
        if t.dtype != torch.int32 or not t.is_cuda or not t.is_contiguous() or t.numel() < size:
            raise ValueError(f"{what}: expected a contiguous CUDA int32 tensor of >= {size} entries")
        if t.device != target.device:
            raise ValueError(f"{what}: must be on the target's device {target.device}")
    st = stream if stream is not None else torch.cuda.current_stream(target.device)
    o = (C.c_float * 3)(*[float(x) for x in origin])
    d = (C.c_int32 * 3)(*[int(x) for x in dims])
    with torch.cuda.device(target.device):   # the library works on the current device
        r = lib.vicp_offsets_static(C.c_void_p(target.data_ptr()), n, o, float(voxel_size), d,
                                    C.c_void_p(keys.data_ptr()), C.c_void_p(offsets.data_ptr()),
                                    C.c_void_p(st.cuda_stream))
    if r != VICP_OK:
        raise VicpError(r, f"vicp_offsets_static: {lib.vicp_status_string(r).decode()} (static scratch holds at "
                           f"most {VICP_STATIC_MAX_VOXELS} voxels and {VICP_STATIC_MAX_BRICK_SLOTS} brick slots)")
    return keys, offsets


def vicp_voxel_histogram(target, origin, voxel_size: float, dims, method: int = VICP_HIST_WARP_AGGREGATED,
                         keys=None, counts=None, stream=None):
    """Voxel keys and per-voxel counts of `target` on an explicit grid by one
    of the two histogram designs (see include/vicp.h).  `counts` (int32[V],
    holding uint32) is added to; it is zeroed here only when not given.
    Returns (keys, counts)."""
    lib = load_library()
    _cloud(target, "target")
    n = target.shape[0]
    V = int(dims[0]) * int(dims[1]) * int(dims[2])
    if keys is None:
        keys = torch.empty(n, dtype=torch.int32, device=target.device)
    if counts is None:
        counts = torch.zeros(V, dtype=torch.int32, device=target.device)
    for t, size, what in ((keys, n, "keys"), (counts, V, "counts")):
        if t.dtype != torch.int32 or not t.is_cuda or not t.is_contiguous() or t.numel() < size:
            raise ValueError(f"{what}: expected a contiguous CUDA int32 tensor of >= {size} entries")
    st = stream if stream is not None else torch.cuda.current_stream(target.device)
    o = (C.c_float * 3)(*[float(x) for x in origin])
    d = (C.c_int32 * 3)(*[int(x) for x in dims])
    r = lib.vicp_voxel_histogram(C.c_void_p(target.data_ptr()), n, o, float(voxel_size), d, int(method),
                                 C.c_void_p(keys.data_ptr()), C.c_void_p(counts.data_ptr()),
                                 C.c_void_p(st.cuda_stream))
    if r != VICP_OK:
        raise VicpError(r, f"vicp_voxel_histogram: {lib.vicp_status_string(r).decode()}")
    return keys, counts


# --- batched registration ---------------------------------------------------
def batch_default_params(**overrides) -> vicp_batch_params:
    p = vicp_batch_params()
    load_library().vicp_batch_default_params(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _sizes(n, P=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(n, dtype=np.int32))
    if a.ndim != 1 or (P is not None and a.shape[0] != P):
        raise ValueError("per-pair sizes: expected a 1-D int32 array with one entry per pair")
    return a


class Batch:
    """A batched-registration context (vicp_batch_*) on the current CUDA
    device and torch stream.  Clouds are pooled: one (sum n, 4) float32
    tensor per side, pair k's rows following pair k-1's."""

    def __init__(self, params: vicp_batch_params | None = None, stream: torch.cuda.Stream | None = None,
                 allocator: vicp_allocator | None = None, **overrides):
        self._lib = load_library()
        self.params = params if params is not None else batch_default_params(**overrides)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._allocator = allocator
        h = C.c_void_p()
        st = self._lib.vicp_batch_create(C.byref(h), C.byref(self.params),
                                         C.byref(allocator) if allocator is not None else None,
                                         C.c_void_p(self.stream.cuda_stream))
        if st != VICP_OK:
            raise VicpError(st, "vicp_batch_create failed")
        self.handle = h
        self.n_pairs = 0

    def _check(self, st: int, what: str):
        if st != VICP_OK:
            raise VicpError(st, f"{what}: {self._lib.vicp_batch_last_error(self.handle).decode()}")

    def close(self):
        if getattr(self, "handle", None):
            self._lib.vicp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def build(self, target: torch.Tensor, n_tgt, voxel_size=None, grid_divisions=None):
        t = _cloud(target, "target")
        n = _sizes(n_tgt)
        P = n.shape[0]
        if int(n.sum()) != t.shape[0]:
            raise ValueError("target rows must equal the sum of n_tgt")
        vs = None if voxel_size is None else np.ascontiguousarray(np.asarray(voxel_size, np.float32))
        dv = None if grid_divisions is None else _sizes(grid_divisions, P)
        for a in (vs, dv):
            if a is not None and a.shape != (P,):
                raise ValueError("per-pair parameters need one entry per pair")
        self._target = t   # the grids refer to it until the next build
        self._check(self._lib.vicp_batch_build(self.handle, P, t.data_ptr(), _ptr(n),
                                               None if vs is None else _ptr(vs),
                                               None if dv is None else _ptr(dv)), "vicp_batch_build")
        self.n_pairs = P

    def register(self, source: torch.Tensor, n_src, poses=None):
        """Returns (status, poses (P, 4, 4) float64, iters (P,), rmse (P,), per-pair status (P,))."""
        s = _cloud(source, "source")
        n = _sizes(n_src, self.n_pairs or None)   # before a build the library reports the call order
        if int(n.sum()) != s.shape[0]:
            raise ValueError("source rows must equal the sum of n_src")
        P = n.shape[0]
        T = np.ascontiguousarray(np.tile(np.eye(4), (P, 1, 1)) if poses is None else poses,
                                 dtype=np.float64).copy()
        it = np.zeros(P, np.int32)
        rm = np.zeros(P, np.float64)
        ps = np.zeros(P, np.int32)
        st = self._lib.vicp_batch_register(self.handle, s.data_ptr(), _ptr(n), _ptr(T), _ptr(it), _ptr(rm), _ptr(ps))
        return st, T, it, rm, ps

    def register_host(self, source, n_src, target, n_tgt, voxel_size=None, grid_divisions=None, poses=None):
        s, t = _host_cloud(source), _host_cloud(target)
        ns, nt = _sizes(n_src), _sizes(n_tgt)
        P = ns.shape[0]
        vs = None if voxel_size is None else np.ascontiguousarray(np.asarray(voxel_size, np.float32))
        dv = None if grid_divisions is None else _sizes(grid_divisions, P)
        T = np.ascontiguousarray(np.tile(np.eye(4), (P, 1, 1)) if poses is None else poses,
                                 dtype=np.float64).copy()
        it = np.zeros(P, np.int32)
        rm = np.zeros(P, np.float64)
        ps = np.zeros(P, np.int32)
        st = self._lib.vicp_batch_register_host(self.handle, P, _ptr(s), _ptr(ns), _ptr(t), _ptr(nt),
                                                None if vs is None else _ptr(vs), None if dv is None else _ptr(dv),
                                                _ptr(T), _ptr(it), _ptr(rm), _ptr(ps))
        if st == VICP_OK:
            self.n_pairs = P
        return st, T, it, rm, ps

    def correspond(self, source: torch.Tensor, n_src, poses: torch.Tensor):
        s = _cloud(source, "source")
        n = _sizes(n_src, self.n_pairs)
        if (poses.dtype != torch.float64 or not poses.is_cuda or poses.numel() != 16 * self.n_pairs
                or not poses.is_contiguous()):
            raise ValueError("poses: contiguous CUDA float64 tensor with 16 entries per pair")
        m = s.shape[0]
        nn = torch.empty(m, dtype=torch.int32, device=s.device)
        d2 = torch.empty(m, dtype=torch.float32, device=s.device)
        self._check(self._lib.vicp_batch_correspond(self.handle, s.data_ptr(), _ptr(n), poses.data_ptr(),
                                                    nn.data_ptr(), d2.data_ptr()), "vicp_batch_correspond")
        return nn, d2

    def tune(self, source: torch.Tensor, n_src, poses=None, iters: int = 4, trials: int = 2):
        s = _cloud(source, "source")
        n = _sizes(n_src, self.n_pairs)
        P = self.n_pairs
        T = np.ascontiguousarray(np.tile(np.eye(4), (P, 1, 1)) if poses is None else poses, dtype=np.float64)
        shape = C.c_int32(-1)
        ms = np.zeros(VICP_BATCH_SHAPES, np.float32)
        self._check(self._lib.vicp_batch_tune(self.handle, s.data_ptr(), _ptr(n), _ptr(T), int(iters), int(trials),
                                              C.byref(shape), _ptr(ms)), "vicp_batch_tune")
        return int(shape.value), ms

    def pair_grid(self, pair: int) -> dict:
        """Copies of pair `pair`'s grid arrays (offsets are pooled positions;
        ids / csr_points are the pair's own segment of the pooled store)."""
        v = vicp_grid_view()
        self._check(self._lib.vicp_batch_pair_grid(self.handle, int(pair), C.byref(v)), "vicp_batch_pair_grid")
        V, n, ns = int(v.n_voxels), int(v.n_target), int(v.n_stored)
        d = self.device
        off = _view(v.offsets, (V + 1,), "<u4", torch.uint32, d).clone()
        base = int(off[0].item()) if V >= 0 else 0
        ids_all = _view(v.ids, (base + ns,), "<i4", torch.int32, d)
        pts_all = _view(v.csr_points, (base + ns, 4), "<f4", torch.float32, d)
        return {
            "origin": tuple(float(v.origin[a]) for a in range(3)), "voxel_size": float(v.voxel_size),
            "inv_voxel_size": float(v.inv_voxel_size), "dims": tuple(int(v.dims[a]) for a in range(3)),
            "n_voxels": V, "n_target": n, "n_stored": ns, "dilation_layers": int(v.dilation_layers),
            "base": base,
            "keys": _view(v.keys, (n,), "<i4", torch.int32, d).clone(),
            "offsets": off,
            "ids": ids_all[base:].clone(),
            "csr_points": pts_all[base:].clone(),
            "occupancy": _view(v.occupancy, ((V + 31) // 32,), "<u4", torch.uint32, d).clone(),
            "root": _view(v.root, (V,), "<i4", torch.int32, d).clone(),
            "ring": _view(v.ring, (V,), "|u1", torch.uint8, d).clone(),
        }

    def report(self, reset: bool = False) -> dict:
        cur, peak = C.c_uint64(0), C.c_uint64(0)
        st = vicp_stats()
        self._check(self._lib.vicp_batch_report(self.handle, C.byref(cur), C.byref(peak), C.byref(st),
                                                1 if reset else 0), "vicp_batch_report")
        out = {name: int(getattr(st, name)) for name, _ in vicp_stats._fields_}
        out.update(current_bytes=int(cur.value), peak_bytes=int(peak.value))
        return out

    def launch_count(self) -> int:
        return int(self._lib.vicp_batch_launch_count(self.handle))

    def graph_replayed(self) -> int:
        """1: the last registration replayed the captured CUDA graph; 0: it
        launched the iterations one by one; -1: no registration yet."""
        return int(self._lib.vicp_batch_graph_replayed(self.handle))

    def set_flags(self, flags: int):
        self._check(self._lib.vicp_batch_set_flags(self.handle, int(flags)), "vicp_batch_set_flags")
        self.params.flags = int(flags)

    def loss(self, source: torch.Tensor, n_src, poses: torch.Tensor, nn: torch.Tensor, dloss=None,
             grad_pose: bool = False, grad_src: bool = False):
        """Per-pair loss (P,) float64 of Eq. 1 at `poses` with the fixed
        correspondences `nn`; with grad_pose the left-perturbation gradients
        (P, 6) float64, with grad_src the per-point gradients (M, 4) float32,
        each weighted by dloss (P,) float64 when given."""
        s = _cloud(source, "source")
        n = _sizes(n_src, self.n_pairs)
        P = self.n_pairs
        if (poses.dtype != torch.float64 or not poses.is_cuda or poses.numel() != 16 * P
                or not poses.is_contiguous()):
            raise ValueError("poses: contiguous CUDA float64 tensor with 16 entries per pair")
        if nn.dtype != torch.int32 or not nn.is_cuda or nn.numel() != s.shape[0] or not nn.is_contiguous():
            raise ValueError("nn: contiguous CUDA int32 tensor with one entry per source point")
        if dloss is not None and (dloss.dtype != torch.float64 or not dloss.is_cuda or dloss.numel() != P
                                  or not dloss.is_contiguous()):
            raise ValueError("dloss: contiguous CUDA float64 tensor with one entry per pair")
        out = torch.empty(P, dtype=torch.float64, device=s.device)
        gp = torch.empty((P, 6), dtype=torch.float64, device=s.device) if grad_pose else None
        gs = torch.empty((s.shape[0], 4), dtype=torch.float32, device=s.device) if grad_src else None
        self._check(self._lib.vicp_batch_loss(self.handle, s.data_ptr(), _ptr(n), poses.data_ptr(), nn.data_ptr(),
                                              None if dloss is None else dloss.data_ptr(), out.data_ptr(),
                                              None if gp is None else gp.data_ptr(),
                                              None if gs is None else gs.data_ptr()), "vicp_batch_loss")
        return out, gp, gs


def vicp_batch_shape_info(shape: int):
    """(threads per block, source points per thread, resident blocks) of an
    iteration kernel shape."""
    th, ppt, rb = C.c_int32(0), C.c_int32(0), C.c_int32(0)
    st = load_library().vicp_batch_shape_info(int(shape), C.byref(th), C.byref(ppt), C.byref(rb))
    if st != VICP_OK:
        raise VicpError(st, f"vicp_batch_shape_info: no shape {shape}")
    return int(th.value), int(ppt.value), int(rb.value)


def vicp_batch_create(params: vicp_batch_params | None = None, stream=None, allocator=None, **overrides) -> Batch:
    return Batch(params, stream, allocator, **overrides)


def vicp_batch_destroy(b: Batch):
    b.close()


def vicp_batch_build(b: Batch, target, n_tgt, voxel_size=None, grid_divisions=None):
    b.build(target, n_tgt, voxel_size, grid_divisions)


def vicp_batch_register(b: Batch, source, n_src, poses=None):
    return b.register(source, n_src, poses)


def vicp_batch_register_host(b: Batch, source, n_src, target, n_tgt, voxel_size=None, grid_divisions=None,
                             poses=None):
    return b.register_host(source, n_src, target, n_tgt, voxel_size, grid_divisions, poses)


def vicp_batch_correspond(b: Batch, source, n_src, poses):
    return b.correspond(source, n_src, poses)


def vicp_batch_tune(b: Batch, source, n_src, poses=None, iters: int = 4, trials: int = 2):
    return b.tune(source, n_src, poses, iters, trials)


def vicp_batch_pair_grid(b: Batch, pair: int) -> dict:
    return b.pair_grid(pair)


# --- differentiable loss -----------------------------------------------------
def _f64_dev(t: torch.Tensor, n: int, what: str):
    if t.dtype != torch.float64 or not t.is_cuda or t.numel() != n or not t.is_contiguous():
        raise ValueError(f"{what}: contiguous CUDA float64 tensor with {n} entries")
    return t


def vicp_se3_exp(xi: torch.Tensor, T0: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    """T = Exp(xi) T0 for (n, 6) xi and (n, 4, 4) T0 (float64, CUDA)."""
    n = xi.shape[0]
    _f64_dev(xi, 6 * n, "xi")
    _f64_dev(T0, 16 * n, "T0")
    out = torch.empty_like(T0) if out is None else _f64_dev(out, 16 * n, "out")
    st = torch.cuda.current_stream(xi.device).cuda_stream
    r = load_library().vicp_se3_exp(n, xi.data_ptr(), T0.data_ptr(), out.data_ptr(), C.c_void_p(st))
    if r != VICP_OK:
        raise VicpError(r, "vicp_se3_exp")
    return out


def vicp_se3_left_jacobian_t(xi: torch.Tensor, g: torch.Tensor) -> torch.Tensor:
    """J(xi)^T g per row, J the left Jacobian of SE(3)."""
    n = xi.shape[0]
    _f64_dev(xi, 6 * n, "xi")
    _f64_dev(g, 6 * n, "g")
    out = torch.empty_like(g)
    st = torch.cuda.current_stream(xi.device).cuda_stream
    r = load_library().vicp_se3_left_jacobian_t(n, xi.data_ptr(), g.data_ptr(), out.data_ptr(), C.c_void_p(st))
    if r != VICP_OK:
        raise VicpError(r, "vicp_se3_left_jacobian_t")
    return out


class PointToPointLoss(torch.autograd.Function):
    """Per-pair loss L_k = (1/M) sum |T p_i - q_nn(i)|^2 (Eq. 1) of a built
    batch at T = Exp(xi) T0, the correspondences from the localised NNS at T
    held fixed.  Differentiable in xi ((P, 6), translation part first) and
    in the source points ((M, 4); the w column gets no gradient).  With
    recompute=True the correspondences are not kept between forward and
    backward but searched again (same poses, the same result)."""

    @staticmethod
    def forward(ctx, xi, source, batch, n_src, T0, recompute=False):
        xi64 = xi.detach().to(torch.float64).contiguous()
        T = vicp_se3_exp(xi64, T0)
        src = source.detach()
        nn, _ = batch.correspond(src, n_src, T)
        loss, _, _ = batch.loss(src, n_src, T, nn)
        ctx.batch, ctx.n_src, ctx.recompute = batch, n_src, recompute
        ctx.xi_dtype = xi.dtype
        if recompute:
            del nn
            ctx.save_for_backward(xi64, T, src)
        else:
            ctx.save_for_backward(xi64, T, src, nn)
        return loss

    @staticmethod
    def backward(ctx, dloss):
        if ctx.recompute:
            xi64, T, src = ctx.saved_tensors
            nn, _ = ctx.batch.correspond(src, ctx.n_src, T)
        else:
            xi64, T, src, nn = ctx.saved_tensors
        dl = dloss.detach().to(torch.float64).contiguous()
        _, g_left, g_src = ctx.batch.loss(src, ctx.n_src, T, nn, dloss=dl, grad_pose=ctx.needs_input_grad[0],
                                          grad_src=ctx.needs_input_grad[1])
        g_xi = vicp_se3_left_jacobian_t(xi64, g_left).to(ctx.xi_dtype) if g_left is not None else None
        return g_xi, g_src, None, None, None, None


def point_to_point_loss(xi, source, batch: Batch, n_src, T0, recompute: bool = False):
    return PointToPointLoss.apply(xi, source, batch, n_src, T0, recompute)
