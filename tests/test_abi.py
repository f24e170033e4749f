"""Host-only checks of the C-ABI library: it builds, loads and exports every
entry point include/fdtd_llg.h declares; argument errors that need no GPU."""
import ctypes as C
import os
import re

import pytest

import paper_2510_22221_b300 as pkg
from paper_2510_22221_b300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = ""
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            text += open(os.path.join(ROOT, "include", f)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fdtd_llg_\w+)\s*\(", text)))


def test_header_and_binding_agree():
    decl = declared_functions()
    assert len(decl) >= 20
    assert set(decl) == set(_abi.SIGNATURES), set(decl) ^ set(_abi.SIGNATURES)


def test_library_exports_every_declared_symbol():
    lib = pkg.load_library()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert lib.fdtd_llg_abi_version() == 2


def test_argument_errors_without_gpu():
    lib = pkg.load_library()
    h = C.c_void_p()
    assert lib.fdtd_llg_create(None, C.byref(h)) == -1
    cfg = _abi.Config()
    cfg.nx, cfg.ny, cfg.nz = 0, 4, 4
    cfg.dx = cfg.dy = cfg.dz = 1e-6
    cfg.courant_factor = 0.5
    assert lib.fdtd_llg_create(C.byref(cfg), C.byref(h)) == -1
    assert b"nx" in lib.fdtd_llg_last_error(None)
    cfg.nx = 4
    cfg.dt = 1.0                      # far above the Courant limit
    assert lib.fdtd_llg_create(C.byref(cfg), C.byref(h)) == -4
    cfg.dt = 0.0
    cfg.courant_factor = 1.5
    assert lib.fdtd_llg_create(C.byref(cfg), C.byref(h)) == -1
    assert lib.fdtd_llg_step(None, 1) == -1
    assert lib.fdtd_llg_sync(None) == -1
    lib.fdtd_llg_destroy(None)


def test_python_layer_has_no_cpu_fallback():
    import torch

    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(RuntimeError):
        pkg.FdtdLlg.create(4, 4, 4, 1e-6, 1e-6, 1e-6)


def test_product_package_does_not_import_oracle():
    pkg_dir = os.path.join(ROOT, "paper_2510_22221_b300")
    for dirpath, _, files in os.walk(pkg_dir):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "yee_llg_oracle" not in src, f


def test_surrogate_argument_errors_without_gpu():
    """The surrogate's entry points refuse bad shapes before touching a GPU."""
    lib = pkg.load_library()
    assert lib.fdtd_llg_lem_param_count(64, 2) == 4 * (4 * 64 * 64 + 4 * 64) + 4 * 64 * (2 + 64 + 2 + 64) + 2 * 64
    assert lib.fdtd_llg_lem_param_count(48, 2) == 0 and lib.fdtd_llg_lem_param_count(64, 5) == 0
    s = _abi.LemShape()
    s.d, s.m, s.batch, s.t_in, s.t_out, s.dt = 64, 2, 512, 200, 400, 1.0
    n = C.c_size_t()
    assert lib.fdtd_llg_lem_workspace_bytes(C.byref(s), C.byref(n)) == 0 and n.value > 0
    s.d = 40
    assert lib.fdtd_llg_lem_workspace_bytes(C.byref(s), C.byref(n)) == -1
    assert b"shape" in lib.fdtd_llg_last_error(None)
    s.d, s.dt = 64, 0.0
    assert lib.fdtd_llg_lem_forward(C.byref(s), None, None, None, None) == -1
    assert lib.fdtd_llg_lem_adam(0, None, None, None, None, 1e-3, 0.9, 0.999, 1e-8, 1, None) == -1
