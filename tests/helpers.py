"""Shared test helpers: build the oracle and the CUDA solver from one workload,
and map between the oracle's full staggered arrays and the library's compact
arrays."""
import os

import numpy as np

import oracle
from oracle import Material as OMaterial, OracleSim, Pml as OPml, Source as OSource


def oracle_from_workload(w, llg_tol=1e-6, llg_max_iter=50, llg_fixed_iter=0, dt=None):
    if dt is None:
        dt = oracle.courant_dt(w.dx, w.dy, w.dz, w.courant)
    mats = [OMaterial(**m) for m in w.materials]
    srcs = [OSource(comp=s["comp"], ijk=(s["i"], s["j"], s["k"]), J0=s["J0"], f0=s["f0"], Tp=s["Tp"], tpk=s["tpk"])
            for s in w.sources]
    eps = w.eps_r_cell() if w.eps_design is not None else None
    pml = None
    if getattr(w, "pml", None):
        q = w.pml
        pml = OPml(n=tuple(q["layers"]), order=q["order"], scale=q["scale"], kappa_max=q["kappa_max"],
                   alpha_max=q["alpha_max"])
    return OracleSim(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, dt, mats, w.mat_id, w.hbias, sources=srcs, probes=w.probes,
                     eps_r_cell=eps, llg_tol=llg_tol, llg_max_iter=llg_max_iter, llg_fixed_iter=llg_fixed_iter,
                     pml=pml)


def compact(sim_oracle):
    """Oracle staggered arrays -> the library's compact (nz, ny, nx) arrays plus
    the three far-wall normal-H arrays."""
    o = sim_oracle
    nx, ny, nz = o.nx, o.ny, o.nz
    out = {
        "Ex": o.Ex[:nz, :ny, :nx], "Ey": o.Ey[:nz, :ny, :nx], "Ez": o.Ez[:nz, :ny, :nx],
        "Hx": o.Hx[:nz, :ny, :nx], "Hy": o.Hy[:nz, :ny, :nx], "Hz": o.Hz[:nz, :ny, :nx],
        "Mx": o.M[0], "My": o.M[1], "Mz": o.M[2],
        "Hx_wall": o.Hx[:, :, nx], "Hy_wall": o.Hy[:, ny, :], "Hz_wall": o.Hz[nz, :, :],
    }
    return {k: np.ascontiguousarray(v) for k, v in out.items()}


def dropped_values(sim_oracle):
    """Largest magnitude among staggered entries the compact layout does not
    hold (E in the far walls): must be zero for the mapping to be lossless."""
    o = sim_oracle
    nx, ny, nz = o.nx, o.ny, o.nz
    parts = [o.Ex[nz], o.Ex[:, ny], o.Ey[nz], o.Ey[:, :, nx], o.Ez[:, ny], o.Ez[:, :, nx]]
    return max(float(np.abs(p).max()) for p in parts)


# Measured errors of the parity tests (GPU against the FP64 oracle), with the
# bound each was checked against; written out at the end of the session to the
# file named by FDTD_PARITY_LOG (JSON lines), if that variable is set.
PARITY_LOG = []


def record(quantity, measured, bound, **extra):
    test = os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0]
    PARITY_LOG.append(dict(test=test, quantity=quantity, measured=float(measured), bound=float(bound), **extra))
