"""ctypes declarations of the C ABI in include/fdtd_llg.h and include/lem_surrogate.h
(marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

from . import _build

FDTD_OK = 0
ERRORS = {
    -1: "FDTD_E_INVAL", -2: "FDTD_E_CUDA", -3: "FDTD_E_OOM", -4: "FDTD_E_UNSTABLE",
    -5: "FDTD_E_LLG_NOCONV", -6: "FDTD_E_STATE", -7: "FDTD_E_RANGE", -8: "FDTD_E_NOSYS",
}
FIELDS = {"Ex": 0, "Ey": 1, "Ez": 2, "Hx": 3, "Hy": 4, "Hz": 5, "Mx": 6, "My": 7, "Mz": 8,
          "Hx_wall": 9, "Hy_wall": 10, "Hz_wall": 11, "dMx": 12, "dMy": 13, "dMz": 14}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Config(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
        ("dt", C.c_double), ("courant_factor", C.c_double), ("llg_tol", C.c_double),
        ("llg_max_iter", C.c_int32), ("llg_fixed_iter", C.c_int32),
        ("probe_capacity", C.c_int32), ("energy_every", C.c_int32), ("device", C.c_int32),
        ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p),
    ]


class MaterialC(C.Structure):
    _fields_ = [("eps_r", C.c_double), ("sigma", C.c_double), ("Ms", C.c_double), ("alpha", C.c_double),
                ("gamma", C.c_double), ("is_pec", C.c_int32), ("pad_", C.c_int32)]


class Profile(C.Structure):
    _fields_ = [("launches", C.c_int64 * 3), ("ms", C.c_double * 3), ("cells", C.c_int64)]


class LemShape(C.Structure):
    _fields_ = [("d", C.c_int32), ("m", C.c_int32), ("batch", C.c_int32), ("t_in", C.c_int32),
                ("t_out", C.c_int32), ("dt", C.c_float)]


class LemPhysics(C.Structure):
    _fields_ = [("lam", C.c_float), ("kappa", C.c_float), ("alpha", C.c_float), ("h0", C.c_float)]


class LLGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None
_vp = C.c_void_p
_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)

# name -> (restype, argtypes) for every entry point declared in include/fdtd_llg.h
SIGNATURES = {
    "fdtd_llg_create": (C.c_int, [C.POINTER(Config), C.POINTER(_vp)]),
    "fdtd_llg_create_batch": (C.c_int, [C.POINTER(Config), C.c_int32, C.POINTER(_vp)]),
    "fdtd_llg_batch_member": (C.c_int, [_vp, C.c_int32, C.POINTER(_vp)]),
    "fdtd_llg_set_materials": (C.c_int, [_vp, _vp, C.POINTER(MaterialC), C.c_int32, _dp, _dp, C.POINTER(C.c_int32)]),
    "fdtd_llg_set_pml": (C.c_int, [_vp, C.POINTER(C.c_int32), C.c_double, C.c_double, C.c_double, C.c_double]),
    "fdtd_llg_set_source": (C.c_int, [_vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_double,
                                      C.c_double, C.c_double]),
    "fdtd_llg_add_probe": (C.c_int, [_vp, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_int32)]),
    "fdtd_llg_step": (C.c_int, [_vp, C.c_int64]),
    "fdtd_llg_sync": (C.c_int, [_vp]),
    "fdtd_llg_probe": (C.c_int, [_vp, C.c_int32, _dp, C.c_int64, _i64p]),
    "fdtd_llg_energy": (C.c_int, [_vp, _dp, C.c_int64, _i64p]),
    "fdtd_llg_time_state": (C.c_int, [_vp, _i64p, C.POINTER(C.c_int32)]),
    "fdtd_llg_get_field": (C.c_int, [_vp, C.c_int32, C.POINTER(C.c_float), C.c_size_t]),
    "fdtd_llg_div_b": (C.c_int, [_vp, _dp, C.c_size_t]),
    "fdtd_llg_set_field": (C.c_int, [_vp, C.c_int32, C.POINTER(C.c_float), C.c_size_t]),
    "fdtd_llg_planes": (C.c_int, [_vp, C.c_int32, C.c_int32, C.POINTER(C.c_float), C.c_size_t, C.c_int32]),
    "fdtd_llg_planes_device": (C.c_int, [_vp, C.c_int32, C.c_int32, _vp, C.c_size_t, C.c_int32]),
    "fdtd_llg_save_state": (C.c_int, [_vp, _vp, C.POINTER(C.c_size_t)]),
    "fdtd_llg_load_state": (C.c_int, [_vp, _vp, C.c_size_t]),
    "fdtd_llg_set_profiling": (C.c_int, [_vp, C.c_int32]),
    "fdtd_llg_read_profile": (C.c_int, [_vp, C.POINTER(Profile), C.c_int32]),
    "fdtd_llg_get_dt": (C.c_int, [_vp, _dp]),
    "fdtd_llg_set_graphs": (C.c_int, [_vp, C.c_int32]),
    "fdtd_llg_set_magnet_cluster": (C.c_int, [_vp, C.c_int32]),
    "fdtd_llg_test_wait_timeout": (C.c_int, [_vp, C.c_int32]),
    "fdtd_llg_get_magnet_cluster": (C.c_int, [_vp, C.POINTER(C.c_int32)]),
    "fdtd_llg_set_tiling": (C.c_int, [_vp, C.c_int32]),
    "fdtd_llg_get_tiling": (C.c_int, [_vp, C.POINTER(C.c_int32)]),
    "fdtd_llg_autotune": (C.c_int, [_vp, C.c_int32, C.POINTER(C.c_int32)]),
    "fdtd_llg_run_checkpointed": (C.c_int, [_vp, C.c_int64, C.c_int32]),
    "fdtd_llg_set_tape_budget": (C.c_int, [_vp, C.c_int64]),
    "fdtd_llg_read_last": (C.c_int, [_vp, _dp, _dp]),
    "fdtd_llg_set_tile_width": (C.c_int, [_vp, C.c_int32]),
    "fdtd_llg_get_tile_width": (C.c_int, [_vp, C.POINTER(C.c_int32)]),
    "fdtd_llg_stream_results": (C.c_int, [_vp, _dp, _dp, C.c_int64]),
    "fdtd_llg_adjoint_step": (C.c_int, [_vp, _dp, _dp, _dp]),
    "fdtd_llg_probe_spectrum": (C.c_int, [_vp, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_int32, C.c_int32,
                                         _dp]),
    "fdtd_llg_fit_modes": (C.c_int, [_dp, C.c_int64, C.c_double, C.c_int32, C.c_int32, C.c_int32, C.c_double,
                                    C.c_double, C.c_int32, _dp, _dp, _dp, _dp, C.POINTER(C.c_int32)]),
    "fdtd_llg_fit_coupling": (C.c_int, [_dp, _dp, C.c_int32, _dp, _dp]),
    "fdtd_llg_e_push_noalloc": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, C.c_int32, C.c_int32, C.c_int32,
                                         C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                         _vp, _vp]),
    "fdtd_llg_lem_param_count": (C.c_longlong, [C.c_int32, C.c_int32]),
    "fdtd_llg_lem_workspace_bytes": (C.c_int, [C.POINTER(LemShape), C.POINTER(C.c_size_t)]),
    "fdtd_llg_lem_views": (C.c_int, [C.POINTER(LemShape), _vp, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp),
                                     C.POINTER(_vp)]),
    "fdtd_llg_lem_forward": (C.c_int, [C.POINTER(LemShape), _vp, _vp, _vp, _vp]),
    "fdtd_llg_lem_loss": (C.c_int, [C.POINTER(LemShape), C.POINTER(LemPhysics), _vp, _vp, _vp, _vp, _vp]),
    "fdtd_llg_lem_backward": (C.c_int, [C.POINTER(LemShape), _vp, _vp, _vp, _vp]),
    "fdtd_llg_lem_adam": (C.c_int, [C.c_longlong, _vp, _vp, _vp, _vp, C.c_float, C.c_float, C.c_float, C.c_float,
                                    C.c_int32, _vp]),
    "fdtd_llg_lem_train_step": (C.c_int, [C.POINTER(LemShape), C.POINTER(LemPhysics), _vp, _vp, _vp, _vp, _vp, _vp,
                                          C.c_float, C.c_int32, _vp, _vp]),
    "fdtd_llg_destroy": (None, [_vp]),
    "fdtd_llg_last_error": (C.c_char_p, [_vp]),
    "fdtd_llg_abi_version": (C.c_int, []),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libfdtd_llg.so.  Raises if it is missing and cannot be built: the
    product has no fallback path."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path) or _build.stale():
            if not build_if_missing:
                raise RuntimeError(f"CUDA library {path} is missing or was built from other sources; "
                                   "run paper_2510_22221_b300._build.build()")
            _build.build()
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(rc: int, handle=None):
    if rc != FDTD_OK:
        msg = load().fdtd_llg_last_error(handle)
        raise LLGError(rc, msg.decode() if msg else "")
