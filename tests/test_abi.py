"""The C ABI library builds for sm_103a, loads without a GPU and exports
exactly the entry points include/vicp.h declares.  Only host-side helpers
that touch no device are called here."""
import ctypes as C
import os
import re

import pytest

from paper_2512_04996_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vicp.h")


def _declared():
    txt = open(HEADER).read()
    return set(re.findall(r"^VICP_API[^(]*?\b(vicp_\w+)\s*\(", txt, flags=re.M))


@pytest.fixture(scope="module")
def lib():
    path = build.build_library()
    return C.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("vicp_create", "vicp_build_grid", "vicp_dilate", "vicp_correspond", "vicp_step",
              "vicp_register", "vicp_destroy", "vicp_get_grid", "vicp_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    pytest.importorskip("torch")
    from paper_2512_04996_gb300 import vicp
    assert set(vicp.SIGNATURES) == _declared()


def test_exports_nothing_undeclared():
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert exported == _declared()


def test_host_only_helpers(lib):
    lib.vicp_abi_version.restype = C.c_int32
    assert lib.vicp_abi_version() == 2
    lib.vicp_status_string.restype = C.c_char_p
    lib.vicp_status_string.argtypes = [C.c_int]
    assert lib.vicp_status_string(7) == b"degenerate geometry"
    lib.vicp_kernel_count.restype = C.c_int32
    lib.vicp_kernel_name.restype = C.c_char_p
    lib.vicp_kernel_name.argtypes = [C.c_int32]
    names = [lib.vicp_kernel_name(i).decode() for i in range(lib.vicp_kernel_count())]
    assert {"histogram", "scan", "brick_scan", "scatter", "dilate", "correspond", "fallback",
            "reduce_solve", "offsets_fill"} <= set(names)


def test_argument_errors_launch_nothing(lib):
    """Bad parameters are rejected before any CUDA call, so this runs on a
    machine without a GPU."""
    pytest.importorskip("torch")
    from paper_2512_04996_gb300 import vicp
    lib2 = vicp.load_library()
    h = C.c_void_p()
    assert lib2.vicp_create(None, None, None, None) == vicp.VICP_ERR_INVALID
    p = vicp.default_params(dilation_layers=32)
    assert lib2.vicp_create(C.byref(h), C.byref(p), None, None) == vicp.VICP_ERR_INVALID
    p = vicp.default_params(grid_divisions=0, voxel_size=0.0)
    assert lib2.vicp_create(C.byref(h), C.byref(p), None, None) == vicp.VICP_ERR_INVALID
    p = vicp.default_params(dims=(4, 0, 4), voxel_size=0.1)
    assert lib2.vicp_create(C.byref(h), C.byref(p), None, None) == vicp.VICP_ERR_INVALID
    assert not h.value
    # every entry point rejects a NULL context
    assert lib2.vicp_build_grid(None, None, 0) == vicp.VICP_ERR_INVALID
    assert lib2.vicp_dilate(None, 3) == vicp.VICP_ERR_INVALID
    assert lib2.vicp_step(None, None, 0, None, None) == vicp.VICP_ERR_INVALID
    assert lib2.vicp_sync(None) == vicp.VICP_ERR_INVALID


def test_default_params_are_the_papers():
    pytest.importorskip("torch")
    import json
    from paper_2512_04996_gb300 import vicp
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_parameters.json")))
    p = vicp.default_params()
    assert p.grid_divisions == 2 ** gold["N"]
    assert p.dilation_layers == gold["dilation_layers"]
    assert p.max_iters == gold["max_iters"]
    assert p.rmse_eps == gold["rmse_eps"]
