"""Binding of the mode fits of the C ABI (ESPRIT on one probe series and the
coupling fit of Eq. omega_pm; arxiv 2510.22221, section "Results").  Argument
marshalling only: the arithmetic is in the library."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _abi
from ._abi import check

_dp = C.POINTER(C.c_double)


def fit_modes(x, dt: float, order: int, pencil: int = 0, fmin: float = 0.0, fmax: float = float("inf"),
              max_modes: int = 8, decimate: int = 1):
    """Modes of a real series by ESPRIT (after block means of `decimate`
    samples): arrays (freq, decay, amp, q) of the up to max_modes strongest
    modes in [fmin, fmax], sorted by frequency."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = [np.zeros(int(max_modes)) for _ in range(4)]
    nfound = C.c_int32(0)
    check(_abi.load().fdtd_llg_fit_modes(x.ctypes.data_as(_dp), x.size, float(dt), int(order), int(pencil),
                                         int(decimate), float(fmin), float(fmax), int(max_modes),
                                         *[o.ctypes.data_as(_dp) for o in out], C.byref(nfound)))
    k = nfound.value
    return tuple(o[:k] for o in out)


def fit_coupling(f_plus, f_minus):
    """(f_p, g) of Eq. omega_pm fitted to hybrid pairs; the splitting at resonance is 2 g."""
    fp = np.ascontiguousarray(f_plus, dtype=np.float64)
    fm = np.ascontiguousarray(f_minus, dtype=np.float64)
    if fp.shape != fm.shape:
        raise ValueError("f_plus and f_minus differ in length")
    a, g = C.c_double(), C.c_double()
    check(_abi.load().fdtd_llg_fit_coupling(fp.ctypes.data_as(_dp), fm.ctypes.data_as(_dp), fp.size, C.byref(a),
                                            C.byref(g)))
    return a.value, g.value
