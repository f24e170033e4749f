"""FP64 CPU oracle of the coupled Yee-Maxwell + LLG step (arxiv 2510.22221,
section "Numerical Model", Eqs. Ampere, Faraday, LLG, llg_tra4-6, iterate_H).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
never does.  It shares no code with the CUDA library.

The arithmetic lives in ``yee_llg_oracle.c`` (plain loops, FP64).  This module
compiles it on demand, marshals numpy arrays into it and exposes a small
``OracleSim`` object.  Closed forms used to pin it are in
``oracle/closed_forms.py``; the brute-force sparse-operator restatement is in
``oracle/operators.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "yee_llg_oracle.c")
_LIB = os.path.join(_HERE, "_yee_llg_oracle.so")


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/_yee_llg_oracle.so`` (gcc, -O2,
    OpenMP over z-planes)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", _LIB + ".tmp", _SRC,
                               "-lm"])
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_u8p = C.POINTER(C.c_uint8)


class _Problem(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("nmat", C.c_int32),
        ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double), ("dt", C.c_double),
        ("mat_eps_r", _dp), ("mat_sigma", _dp), ("mat_Ms", _dp), ("mat_alpha", _dp), ("mat_gamma", _dp),
        ("mat_pec", _ip),
        ("mat_id", _u8p),
        ("eps_r_cell", _dp),
        ("hbias", C.c_double * 3),
        ("nsrc", C.c_int32), ("nprobe", C.c_int32),
        ("src", _ip), ("src_par", _dp), ("probe", _ip),
        ("llg_tol", C.c_double),
        ("llg_max_iter", C.c_int32),
        ("llg_fixed_iter", C.c_int32),
        ("pml_n", C.c_int32 * 3), ("pml_pad_", C.c_int32),
        ("pml_order", C.c_double), ("pml_scale", C.c_double),
        ("pml_kappa_max", C.c_double), ("pml_alpha_max", C.c_double),
    ]


class _State(C.Structure):
    _fields_ = [("Ex", _dp), ("Ey", _dp), ("Ez", _dp), ("Hx", _dp), ("Hy", _dp), ("Hz", _dp),
                ("M", _dp), ("step", C.c_int64), ("psi", _dp)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.orc_run.argtypes = [C.POINTER(_Problem), C.POINTER(_State), C.c_int64, _dp, _dp, _ip]
        _lib.orc_run.restype = C.c_int
        _lib.orc_half_push.argtypes = [C.POINTER(_Problem), C.POINTER(_State)]
        _lib.orc_half_push.restype = C.c_int
        _lib.orc_energy.argtypes = [C.POINTER(_Problem), C.POINTER(_State)]
        _lib.orc_energy.restype = C.c_double
        _lib.orc_div_b.argtypes = [C.POINTER(_Problem), C.POINTER(_State), _dp]
        _lib.orc_div_b.restype = None
        _lib.orc_courant_dt.argtypes = [C.c_double] * 4
        _lib.orc_courant_dt.restype = C.c_double
        _lib.orc_source_value.argtypes = [_dp, C.c_double]
        _lib.orc_source_value.restype = C.c_double
        _lib.orc_llg_trapezoid.argtypes = [_dp, _dp, _dp, C.c_double, C.c_double, C.c_double, _dp]
        _lib.orc_llg_trapezoid.restype = None
        _lib.orc_psi_size.argtypes = [C.POINTER(_Problem)]
        _lib.orc_psi_size.restype = C.c_int64
        _lib.orc_set_threads.argtypes = [C.c_int]
        _lib.orc_set_threads.restype = C.c_int
        # one thread unless asked: the tests run many small problems, and the
        # timed baselines state the count they use
        _lib.orc_set_threads(int(os.environ.get("ORACLE_THREADS", "1")))
        for nm in ("orc_mu0", "orc_eps0", "orc_c0"):
            getattr(_lib, nm).restype = C.c_double
            getattr(_lib, nm).argtypes = []
    return _lib


def set_threads(n: int) -> int:
    """Threads of the oracle's parallel loops (<= 0: every host core); returns
    the count now in use.  Results do not depend on it (see the C header)."""
    return int(lib().orc_set_threads(int(n)))


def _p(a, ct=_dp):
    return a.ctypes.data_as(ct) if a is not None else None


def mu0() -> float:
    return lib().orc_mu0()


def eps0() -> float:
    return lib().orc_eps0()


def c0() -> float:
    return lib().orc_c0()


def courant_dt(dx: float, dy: float, dz: float, cfl: float) -> float:
    """dt = CFL / (c sqrt(1/dx^2 + 1/dy^2 + 1/dz^2)) (section "Modeling Setup")."""
    return lib().orc_courant_dt(dx, dy, dz, cfl)


def source_value(J0: float, f0: float, Tp: float, tpk: float, t: float) -> float:
    """Modulated Gaussian of section "Modeling Setup": exp(-(t-tpk)^2/2Tp^2) cos(2 pi f0 t)."""
    par = np.array([J0, f0, Tp, tpk], dtype=np.float64)
    return lib().orc_source_value(_p(par), t)


def llg_trapezoid(M, He_n, He_np1, kappa, alpha, Ms):
    """One solve of Eqs. llg_tra4-6 with prescribed H_eff at both ends, then |M| = Ms."""
    M = np.ascontiguousarray(M, dtype=np.float64)
    a = np.ascontiguousarray(He_n, dtype=np.float64)
    b = np.ascontiguousarray(He_np1, dtype=np.float64)
    out = np.zeros(3)
    lib().orc_llg_trapezoid(_p(M), _p(a), _p(b), kappa, alpha, Ms, _p(out))
    return out


@dataclass
class Material:
    eps_r: float = 1.0
    sigma: float = 0.0
    Ms: float = 0.0
    alpha: float = 0.0
    gamma: float = 1.76e11       # |gamma| in rad/(s T)
    pec: bool = False


@dataclass
class Pml:
    """Convolutional PML (reading R15 of the oracle: CFS stretch, graded
    sigma, kappa, alpha) in the first and last ``n[a]`` cells of each axis."""
    n: tuple = (8, 8, 8)         # layers per axis (0: none on that axis)
    order: float = 3.0           # grading exponent m
    scale: float = 1.0           # sigma_max / (0.8 (m+1) / (eta0 d))
    kappa_max: float = 1.0
    alpha_max: float = 0.0       # S/m


@dataclass
class Source:
    comp: int                    # 0: Jx on an Ex edge, 1: Jy, 2: Jz
    ijk: tuple
    J0: float
    f0: float
    Tp: float = 0.0              # 0 -> 1/f0 (one period)
    tpk: float = 0.0             # 0 -> 3 Tp


class OracleSim:
    """FP64 state + problem; ``run`` advances full steps in the C oracle.

    Field arrays are numpy float64 with full staggered shapes in (k, j, i)
    order: Ex (nz+1, ny+1, nx), Ey (nz+1, ny, nx+1), Ez (nz, ny+1, nx+1),
    Hx (nz, ny, nx+1), Hy (nz, ny+1, nx), Hz (nz+1, ny, nx), M (3, nz, ny, nx).
    """

    def __init__(self, nx, ny, nz, dx, dy, dz, dt, materials, mat_id, hbias,
                 sources=(), probes=(), eps_r_cell=None, llg_tol=1e-6, llg_max_iter=50,
                 llg_fixed_iter=0, pml=None):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.dx, self.dy, self.dz, self.dt = float(dx), float(dy), float(dz), float(dt)
        self.materials = list(materials)
        self.mat_id = np.ascontiguousarray(mat_id, dtype=np.uint8).reshape(nz, ny, nx)
        self.hbias = np.asarray(hbias, dtype=np.float64).reshape(3)
        self.eps_r_cell = None if eps_r_cell is None else np.ascontiguousarray(eps_r_cell, dtype=np.float64).reshape(nz, ny, nx)
        self._m_eps = np.array([m.eps_r for m in self.materials], dtype=np.float64)
        self._m_sig = np.array([m.sigma for m in self.materials], dtype=np.float64)
        self._m_Ms = np.array([m.Ms for m in self.materials], dtype=np.float64)
        self._m_al = np.array([m.alpha for m in self.materials], dtype=np.float64)
        self._m_ga = np.array([m.gamma for m in self.materials], dtype=np.float64)
        self._m_pec = np.array([1 if m.pec else 0 for m in self.materials], dtype=np.int32)
        srcs = []
        pars = []
        for s in sources:
            Tp = s.Tp if s.Tp > 0 else 1.0 / s.f0
            tpk = s.tpk if s.tpk > 0 else 3.0 * Tp
            srcs.append([s.comp, *s.ijk])
            pars.append([s.J0, s.f0, Tp, tpk])
        self._src = np.array(srcs, dtype=np.int32).reshape(-1, 4)
        self._spar = np.array(pars, dtype=np.float64).reshape(-1, 4)
        self._probe = np.array(list(probes), dtype=np.int32).reshape(-1, 3)
        self.llg_tol, self.llg_max_iter, self.llg_fixed_iter = llg_tol, llg_max_iter, llg_fixed_iter
        self.pml = pml
        n = (self.nx, self.ny, self.nz)
        self.Ex = np.zeros((nz + 1, ny + 1, nx))
        self.Ey = np.zeros((nz + 1, ny, nx + 1))
        self.Ez = np.zeros((nz, ny + 1, nx + 1))
        self.Hx = np.zeros((nz, ny, nx + 1))
        self.Hy = np.zeros((nz, ny + 1, nx))
        self.Hz = np.zeros((nz + 1, ny, nx))
        self.M = np.zeros((3, nz, ny, nx))
        self.step = 0
        # initial magnetisation along the bias (|M| = Ms); z when the bias is zero
        h = np.linalg.norm(self.hbias)
        u = self.hbias / h if h > 0 else np.array([0.0, 0.0, 1.0])
        Ms = self._m_Ms[self.mat_id]
        for d in range(3):
            self.M[d] = Ms * u[d]
        del n
        self.psi = np.zeros(lib().orc_psi_size(C.byref(self._problem()))) if pml is not None else None

    # -- ctypes marshalling
    def _problem(self):
        P = _Problem()
        P.nx, P.ny, P.nz, P.nmat = self.nx, self.ny, self.nz, len(self.materials)
        P.dx, P.dy, P.dz, P.dt = self.dx, self.dy, self.dz, self.dt
        P.mat_eps_r, P.mat_sigma, P.mat_Ms = _p(self._m_eps), _p(self._m_sig), _p(self._m_Ms)
        P.mat_alpha, P.mat_gamma, P.mat_pec = _p(self._m_al), _p(self._m_ga), _p(self._m_pec, _ip)
        P.mat_id = _p(self.mat_id, _u8p)
        P.eps_r_cell = _p(self.eps_r_cell) if self.eps_r_cell is not None else None
        P.hbias[0], P.hbias[1], P.hbias[2] = (float(v) for v in self.hbias)
        P.nsrc, P.nprobe = self._src.shape[0], self._probe.shape[0]
        P.src, P.src_par, P.probe = _p(self._src, _ip), _p(self._spar), _p(self._probe, _ip)
        P.llg_tol, P.llg_max_iter, P.llg_fixed_iter = self.llg_tol, self.llg_max_iter, self.llg_fixed_iter
        if self.pml is not None:
            for a in range(3):
                P.pml_n[a] = int(self.pml.n[a])
            P.pml_order, P.pml_scale = float(self.pml.order), float(self.pml.scale)
            P.pml_kappa_max, P.pml_alpha_max = float(self.pml.kappa_max), float(self.pml.alpha_max)
        return P

    def _state(self):
        for nm in ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz", "M"):
            a = getattr(self, nm)
            if not (a.flags.c_contiguous and a.dtype == np.float64):
                setattr(self, nm, np.ascontiguousarray(a, dtype=np.float64))
        S = _State()
        S.Ex, S.Ey, S.Ez = _p(self.Ex), _p(self.Ey), _p(self.Ez)
        S.Hx, S.Hy, S.Hz = _p(self.Hx), _p(self.Hy), _p(self.Hz)
        S.M, S.step = _p(self.M), self.step
        S.psi = _p(self.psi) if self.psi is not None else None
        return S

    def run(self, nsteps: int):
        """Advance ``nsteps``; returns dict(probes (n, nprobe, 9), energy (n,),
        iters (n, 2), noconv bool)."""
        P, S = self._problem(), self._state()
        npb = max(self._probe.shape[0], 1)
        probes = np.zeros((nsteps, npb, 9))
        energy = np.zeros(nsteps)
        iters = np.zeros((nsteps, 2), dtype=np.int32)
        rc = lib().orc_run(C.byref(P), C.byref(S), nsteps, _p(probes), _p(energy), _p(iters, _ip))
        if rc == -2:
            raise ValueError("PML layers set without their memory")
        if rc < 0:
            raise MemoryError("oracle allocation failed")
        self.step = S.step
        return dict(probes=probes[:, : self._probe.shape[0]], energy=energy, iters=iters, noconv=rc == 1)

    def half_push(self) -> int:
        """Move H, M half a step ahead with the curl of the present E."""
        P, S = self._problem(), self._state()
        return lib().orc_half_push(C.byref(P), C.byref(S))

    def energy(self) -> float:
        P, S = self._problem(), self._state()
        return lib().orc_energy(C.byref(P), C.byref(S))

    def div_b(self) -> np.ndarray:
        """div(H + M_face) at cell centres, shape (nz, ny, nx)."""
        P, S = self._problem(), self._state()
        out = np.zeros((self.nz, self.ny, self.nx))
        lib().orc_div_b(C.byref(P), C.byref(S), _p(out))
        return out

    def psi_blocks(self) -> dict:
        """The PML memories by name ('Ex|y': Ex's memory of d/dy, ...), each in
        its component's staggered shape."""
        names = ["Ex|y", "Ex|z", "Ey|z", "Ey|x", "Ez|x", "Ez|y", "Hx|y", "Hx|z", "Hy|z", "Hy|x", "Hz|x", "Hz|y"]
        out, off = {}, 0
        for nm in names:
            shape = getattr(self, nm[:2]).shape
            sz = int(np.prod(shape))
            out[nm] = self.psi[off: off + sz].reshape(shape)
            off += sz
        return out

    def copy_fields(self) -> dict:
        return {nm: getattr(self, nm).copy() for nm in ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz", "M")}

    def set_fields(self, **kw):
        for nm, v in kw.items():
            cur = getattr(self, nm)
            setattr(self, nm, np.array(np.broadcast_to(v, cur.shape), dtype=np.float64, order="C", copy=True))


__all__ = ["build", "set_threads", "OracleSim", "Material", "Source", "Pml", "courant_dt", "source_value", "llg_trapezoid",
           "mu0", "eps0", "c0"]
