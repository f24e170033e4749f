"""Thin Python binding of the C ABI (include/fdtd_llg.h): argument
marshalling only; every step of the method runs in libfdtd_llg.so.

PyTorch supplies the CUDA stream and, by default, device memory through its
caching allocator (passed to the library as alloc/free callbacks).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import Sequence

import numpy as np

from . import _abi
from ._abi import FIELDS, check


@dataclass
class Material:
    eps_r: float = 1.0
    sigma: float = 0.0
    Ms: float = 0.0            # A/m; 0 = non-magnetic
    alpha: float = 0.0
    gamma: float = 1.76e11     # |gamma| in rad/(s T)
    pec: bool = False


class _TorchAllocator:
    """alloc/free callbacks backed by torch's CUDA caching allocator."""

    def __init__(self):
        import torch

        def _alloc(nbytes, stream, user):
            try:
                # the legacy default stream (handle 1) is torch's default stream (handle 0)
                s = stream if stream not in (None, _LEGACY_STREAM) else 0
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), stream=s))
            except Exception:
                return None

        def _free(ptr, user):
            torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = _abi.ALLOC_FN(_alloc)
        self.free = _abi.FREE_FN(_free)


def _config(nx, ny, nz, dx, dy, dz, dt, courant_factor, llg_tol, llg_max_iter, llg_fixed_iter,
            probe_capacity, energy, device, stream, allocator):
    cfg = _abi.Config()
    cfg.nx, cfg.ny, cfg.nz = int(nx), int(ny), int(nz)
    cfg.dx, cfg.dy, cfg.dz = float(dx), float(dy), float(dz)
    cfg.dt, cfg.courant_factor = float(dt), float(courant_factor)
    cfg.llg_tol, cfg.llg_max_iter, cfg.llg_fixed_iter = float(llg_tol), int(llg_max_iter), int(llg_fixed_iter)
    cfg.probe_capacity, cfg.energy_every, cfg.device = int(probe_capacity), 1 if energy else 0, int(device)
    cfg.stream = stream
    if allocator is not None:
        cfg.alloc, cfg.free = allocator.alloc, allocator.free
    return cfg


_LEGACY_STREAM = 1   # cudaStreamLegacy


def _torch_stream(device):
    """torch's current stream as a cudaStream_t.  torch reports its default
    stream as 0, which the C ABI reads as "create a stream of your own"; the
    explicit legacy-stream handle keeps the work on torch's default stream, so
    events and synchronisation on torch's side see it."""
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the solver runs only on the GPU")
    h = torch.cuda.current_stream(device).cuda_stream
    return h if h else _LEGACY_STREAM


class FdtdLlg:
    """One grid (``create``) or a batch of grids (``create_batch``)."""

    def __init__(self, handle, root, allocator=None, dims=None):
        self._h = handle
        self._root = root          # the owning handle object (self for roots)
        self._alloc = allocator
        self._dims = dims          # (nx, ny, nz)
        self._members = {}
        self._batch_dims = None
        self._probes = 0           # probes added through this instance handle

    # ------------------------------------------------------------- creation
    @classmethod
    def create(cls, nx, ny, nz, dx, dy, dz, dt=0.0, courant_factor=0.5, llg_tol=1e-6, llg_max_iter=20,
               llg_fixed_iter=0, probe_capacity=4096, energy=True, device=0, torch_memory=True):
        lib = _abi.load()
        stream = _torch_stream(device)
        alloc = _TorchAllocator() if torch_memory else None
        cfg = _config(nx, ny, nz, dx, dy, dz, dt, courant_factor, llg_tol, llg_max_iter, llg_fixed_iter,
                      probe_capacity, energy, device, stream, alloc)
        h = C.c_void_p()
        check(lib.fdtd_llg_create(C.byref(cfg), C.byref(h)))
        obj = cls(h, None, alloc, (int(nx), int(ny), int(nz)))
        obj._root = obj
        return obj

    @classmethod
    def create_batch(cls, dims: Sequence[tuple], spacings: Sequence[tuple], dt=0.0, courant_factor=0.5,
                     llg_tol=1e-6, llg_max_iter=20, llg_fixed_iter=0, probe_capacity=4096, energy=True,
                     device=0, torch_memory=True):
        lib = _abi.load()
        stream = _torch_stream(device)
        alloc = _TorchAllocator() if torch_memory else None
        n = len(dims)
        arr = (_abi.Config * n)()
        for q, ((nx, ny, nz), (dx, dy, dz)) in enumerate(zip(dims, spacings)):
            arr[q] = _config(nx, ny, nz, dx, dy, dz, dt, courant_factor, llg_tol, llg_max_iter, llg_fixed_iter,
                             probe_capacity, energy, device, stream, alloc)
        h = C.c_void_p()
        check(lib.fdtd_llg_create_batch(arr, n, C.byref(h)))
        obj = cls(h, None, alloc, None)
        obj._root = obj
        obj._batch_dims = [tuple(int(v) for v in d) for d in dims]
        if n == 1:
            obj._dims = obj._batch_dims[0]
        return obj

    def batch_member(self, i: int) -> "FdtdLlg":
        if self._batch_dims is None:
            if i != 0:
                raise IndexError("a single-instance handle has only member 0")
            return self
        if i not in self._members:
            m = C.c_void_p()
            check(_abi.load().fdtd_llg_batch_member(self._h, int(i), C.byref(m)), self._h)
            self._members[i] = FdtdLlg(m, self, None, self._batch_dims[i])
        return self._members[i]

    # ------------------------------------------------------------ set-up
    def set_materials(self, mat_id, table: Sequence[Material], hbias, eps_r_design=None, design_box=None):
        lib = _abi.load()
        nx, ny, nz = self._dims
        if hasattr(mat_id, "data_ptr"):                      # torch tensor (host or device)
            if mat_id.numel() != nx * ny * nz:
                raise ValueError("mat_id must hold nx*ny*nz entries")
            keep = mat_id.contiguous()
            ptr = C.c_void_p(keep.data_ptr())
        else:
            keep = np.ascontiguousarray(mat_id, dtype=np.uint8).reshape(-1)
            if keep.size != nx * ny * nz:
                raise ValueError("mat_id must hold nx*ny*nz entries")
            ptr = C.c_void_p(keep.ctypes.data)
        tab = (_abi.MaterialC * len(table))()
        for q, m in enumerate(table):
            tab[q] = _abi.MaterialC(m.eps_r, m.sigma, m.Ms, m.alpha, m.gamma, 1 if m.pec else 0, 0)
        hb = (C.c_double * 3)(*[float(v) for v in hbias])
        des = None
        box = None
        des_np = None
        if eps_r_design is not None:
            des_np = np.ascontiguousarray(eps_r_design, dtype=np.float64).reshape(-1)
            des = des_np.ctypes.data_as(C.POINTER(C.c_double))
            box = (C.c_int32 * 6)(*[int(v) for v in design_box])
        rc = lib.fdtd_llg_set_materials(self._h, ptr, tab, len(table), hb, des, box)
        del keep, des_np
        check(rc, self._h)

    def set_pml(self, layers, order=3.0, scale=1.0, kappa_max=1.0, alpha_max=0.0):
        """Absorbing layers (convolutional PML) in the first and last
        ``layers[a]`` cells of axis a; ``(0, 0, 0)`` removes them."""
        arr = (C.c_int32 * 3)(*(int(v) for v in layers))
        check(_abi.load().fdtd_llg_set_pml(self._h, arr, float(order), float(scale), float(kappa_max),
                                           float(alpha_max)), self._h)

    def set_source(self, comp, i, j, k, J0, f0, Tp=0.0, t_peak=0.0):
        check(_abi.load().fdtd_llg_set_source(self._h, int(comp), int(i), int(j), int(k), float(J0), float(f0),
                                              float(Tp), float(t_peak)), self._h)

    def add_probe(self, i, j, k) -> int:
        pid = C.c_int32()
        check(_abi.load().fdtd_llg_add_probe(self._h, int(i), int(j), int(k), C.byref(pid)), self._h)
        self._probes = pid.value + 1
        return pid.value

    # -------------------------------------------------------------- run
    def step(self, nsteps: int):
        check(_abi.load().fdtd_llg_step(self._h, int(nsteps)), self._h)

    def sync(self):
        check(_abi.load().fdtd_llg_sync(self._h), self._h)

    @property
    def dt(self) -> float:
        """Time step (s) of the handle's batch."""
        v = C.c_double()
        check(_abi.load().fdtd_llg_get_dt(self._h, C.byref(v)), self._h)
        return v.value

    def time_state(self):
        s = C.c_int64()
        half = C.c_int32()
        check(_abi.load().fdtd_llg_time_state(self._h, C.byref(s), C.byref(half)), self._h)
        return s.value, bool(half.value)

    # ------------------------------------------------------------ outputs
    def probe(self, pid: int, cap_rows: int = 1 << 40) -> np.ndarray:
        lib = _abi.load()
        step, _ = self.time_state()
        rows_max = int(min(cap_rows, step))
        out = np.zeros((max(rows_max, 1), 9))
        rows = C.c_int64()
        check(lib.fdtd_llg_probe(self._h, int(pid), out.ctypes.data_as(C.POINTER(C.c_double)), rows_max,
                                 C.byref(rows)), self._h)
        return out[: rows.value]

    def energy(self, cap: int = 1 << 40) -> np.ndarray:
        lib = _abi.load()
        step, _ = self.time_state()
        n = int(min(cap, step))
        out = np.zeros(max(n, 1))
        w = C.c_int64()
        check(lib.fdtd_llg_energy(self._h, out.ctypes.data_as(C.POINTER(C.c_double)), n, C.byref(w)), self._h)
        return out[: w.value]

    def read_last(self):
        """(rows, energy) of the newest step: rows (nprobes, 9) for every
        probe, one stream synchronisation."""
        lib = _abi.load()
        rows = np.zeros((max(self._probes, 1), 9))
        e = C.c_double()
        check(lib.fdtd_llg_read_last(self._h, rows.ctypes.data_as(C.POINTER(C.c_double)), C.byref(e)), self._h)
        return rows[: self._probes], e.value

    def stream_results(self, rows=None, energy=None):
        """Stream every following step's probe rows and energy into host
        rings: rows (capacity, nprobes, 9) and energy (capacity,), float64
        numpy arrays or CPU torch tensors (page-locked ones keep the copies
        asynchronous); step n goes to slot n % capacity, complete after the
        next synchronising call.  No arguments stop streaming."""

        def ptr(a):
            if a is None:
                return None, 0
            if hasattr(a, "data_ptr"):
                if a.dtype != __import__("torch").float64 or a.is_cuda or not a.is_contiguous():
                    raise ValueError("host rings must be contiguous float64 CPU tensors")
                return C.cast(a.data_ptr(), C.POINTER(C.c_double)), a.shape[0]
            if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
                raise ValueError("host rings must be contiguous float64 arrays")
            return a.ctypes.data_as(C.POINTER(C.c_double)), a.shape[0]

        pr, cr = ptr(rows)
        pe, ce = ptr(energy)
        if rows is not None and energy is not None and cr != ce:
            raise ValueError("rows and energy rings need the same capacity")
        if rows is not None and tuple(rows.shape[1:]) != (self._probes, 9):
            raise ValueError("rows ring must be (capacity, nprobes, 9)")
        check(_abi.load().fdtd_llg_stream_results(self._h, pr, pe, int(cr or ce)), self._h)
        self._rings = (rows, energy)   # kept alive while the library writes into them

    def _shape(self, name):
        nx, ny, nz = self._dims
        return {"Hx_wall": (nz, ny), "Hy_wall": (nz, nx), "Hz_wall": (ny, nx)}.get(name, (nz, ny, nx))

    def div_b(self) -> np.ndarray:
        """div(H + M_face) at every cell centre of the present state, FP64,
        shape (nz, ny, nx)."""
        n = int(self._dims[0]) * int(self._dims[1]) * int(self._dims[2])
        out = np.zeros(n)
        check(_abi.load().fdtd_llg_div_b(self._h, out.ctypes.data_as(C.POINTER(C.c_double)), n), self._h)
        return out.reshape(self._dims[2], self._dims[1], self._dims[0])

    def get_field(self, name: str) -> np.ndarray:
        shp = self._shape(name)
        out = np.zeros(shp, dtype=np.float32)
        check(_abi.load().fdtd_llg_get_field(self._h, FIELDS[name], out.ctypes.data_as(C.POINTER(C.c_float)),
                                             out.size), self._h)
        return out

    def set_field(self, name: str, values):
        shp = self._shape(name)
        arr = np.ascontiguousarray(np.broadcast_to(values, shp), dtype=np.float32)
        check(_abi.load().fdtd_llg_set_field(self._h, FIELDS[name], arr.ctypes.data_as(C.POINTER(C.c_float)),
                                             arr.size), self._h)

    def read_planes(self, k0: int, k1: int) -> np.ndarray:
        """The stored state of z-planes [k0, k1) as one float32 array (layout
        of fdtd_llg_planes), exact and without changing the time state."""
        nx, ny, _ = self._dims
        out = np.empty((k1 - k0) * (9 * nx * ny + nx + ny), dtype=np.float32)
        check(_abi.load().fdtd_llg_planes(self._h, int(k0), int(k1), out.ctypes.data_as(C.POINTER(C.c_float)),
                                          out.size, 0), self._h)
        return out

    def write_planes(self, k0: int, k1: int, data):
        """Overwrite the stored state of z-planes [k0, k1) with what
        read_planes returned (possibly from another handle's slab)."""
        arr = np.ascontiguousarray(data, dtype=np.float32).reshape(-1)
        check(_abi.load().fdtd_llg_planes(self._h, int(k0), int(k1), arr.ctypes.data_as(C.POINTER(C.c_float)),
                                          arr.size, 1), self._h)

    def plane_floats(self, k0: int, k1: int) -> int:
        """Floats of the stored state of z-planes [k0, k1) (layout of fdtd_llg_planes)."""
        nx, ny, _ = self._dims
        return (k1 - k0) * (9 * nx * ny + nx + ny)

    def read_planes_device(self, k0: int, k1: int, out):
        """Queue on the handle's stream a copy of the stored state of z-planes
        [k0, k1) into `out` (a float32 CUDA tensor of plane_floats elements),
        with no synchronisation."""
        if not (out.is_cuda and out.dtype.is_floating_point and out.element_size() == 4 and out.is_contiguous()):
            raise ValueError("out must be a contiguous float32 CUDA tensor")
        check(_abi.load().fdtd_llg_planes_device(self._h, int(k0), int(k1), C.c_void_p(out.data_ptr()), out.numel(), 0),
              self._h)

    def write_planes_device(self, k0: int, k1: int, data):
        """Queue on the handle's stream the overwrite of z-planes [k0, k1) from
        `data` (a float32 CUDA tensor laid out as read_planes_device writes it)."""
        if not (data.is_cuda and data.element_size() == 4 and data.is_contiguous()):
            raise ValueError("data must be a contiguous float32 CUDA tensor")
        check(_abi.load().fdtd_llg_planes_device(self._h, int(k0), int(k1), C.c_void_p(data.data_ptr()), data.numel(), 1),
              self._h)

    def save_state(self) -> bytes:
        lib = _abi.load()
        n = C.c_size_t()
        check(lib.fdtd_llg_save_state(self._h, None, C.byref(n)), self._h)
        buf = C.create_string_buffer(n.value)
        check(lib.fdtd_llg_save_state(self._h, buf, C.byref(n)), self._h)
        return buf.raw[: n.value]

    def load_state(self, data: bytes):
        buf = C.create_string_buffer(data, len(data))
        check(_abi.load().fdtd_llg_load_state(self._h, buf, len(data)), self._h)

    def probe_spectrum(self, pid: int, comp: int, f0: float, f1: float, nf: int, window: str = "hann") -> np.ndarray:
        """|DFT| of probe `pid`, column `comp` (0-2 E, 3-5 H, 6-8 M), at nf
        frequencies from f0 to f1, computed on the GPU from the device ring."""
        out = np.zeros(int(nf))
        win = {"rect": 0, "hann": 1}[window]
        check(_abi.load().fdtd_llg_probe_spectrum(self._h, int(pid), int(comp), float(f0), float(f1), int(nf), win,
                                                   out.ctypes.data_as(C.POINTER(C.c_double))), self._h)
        return out

    # -------------------------------------------------------------- adjoint
    def run_checkpointed(self, nsteps: int, interval: int = 0):
        """Run nsteps from step 0 keeping sqrt(N)-spaced checkpoints for adjoint()."""
        check(_abi.load().fdtd_llg_run_checkpointed(self._h, int(nsteps), int(interval)), self._h)
        self._adj_steps = int(nsteps)

    def set_tape_budget(self, nbytes: int):
        """Device bytes the next run_checkpointed may spend on records taken
        during the run (< 0: half the free memory, 0: recompute every segment)."""
        check(_abi.load().fdtd_llg_set_tape_budget(self._h, int(nbytes)), self._h)

    def adjoint_step(self, dJ_dE, design_shape=None):
        """Gradients of J given dJ/dE at the probes (nsteps x nprobes x 3):
        (dJ/d eps_r of the design cells or None, dJ/d |H_bias| per A/m)."""
        seed = np.ascontiguousarray(dJ_dE, dtype=np.float64)
        ge = np.zeros(design_shape) if design_shape is not None else None
        gh = C.c_double(0.0)
        check(_abi.load().fdtd_llg_adjoint_step(self._h, seed.ctypes.data_as(C.POINTER(C.c_double)),
                                           ge.ctypes.data_as(C.POINTER(C.c_double)) if ge is not None else None,
                                           C.byref(gh)), self._h)
        return ge, gh.value

    # --------------------------------------------------------------- tiling
    def set_tiling(self, planes: int):
        """z-planes per field-sweep task; 0 lets the library choose."""
        check(_abi.load().fdtd_llg_set_tiling(self._h, int(planes)), self._h)

    def set_graphs(self, mode: int):
        """CUDA graphs for long step calls: 1 on, 0 off, -1 automatic."""
        check(_abi.load().fdtd_llg_set_graphs(self._h, int(mode)), self._h)

    def test_wait_timeout(self, polls: int):
        """Make the first sweep CTA's bounded wait run out (see the header);
        0 turns it off."""
        check(_abi.load().fdtd_llg_test_wait_timeout(self._h, int(polls)), self._h)

    def set_magnet_cluster(self, ctas: int):
        """Magnet CTAs per magnetic region (0: automatic, 1..8)."""
        check(_abi.load().fdtd_llg_set_magnet_cluster(self._h, int(ctas)), self._h)

    def get_magnet_cluster(self) -> int:
        v = C.c_int32()
        check(_abi.load().fdtd_llg_get_magnet_cluster(self._h, C.byref(v)), self._h)
        return v.value

    def set_tile_width(self, width: int):
        """Sweep tile shape: 64 (64 x 8), 32 (32 x 16) or 0 (fewest padded cells)."""
        check(_abi.load().fdtd_llg_set_tile_width(self._h, int(width)), self._h)

    def get_tile_width(self) -> int:
        w = C.c_int32()
        check(_abi.load().fdtd_llg_get_tile_width(self._h, C.byref(w)), self._h)
        return w.value

    def get_tiling(self) -> int:
        p = C.c_int32(0)
        check(_abi.load().fdtd_llg_get_tiling(self._h, C.byref(p)), self._h)
        return p.value

    def autotune(self, trial_steps: int = 20) -> int:
        """Time the candidate tilings with real steps (they advance the run) and keep the fastest."""
        p = C.c_int32(0)
        check(_abi.load().fdtd_llg_autotune(self._h, int(trial_steps), C.byref(p)), self._h)
        return p.value

    # ------------------------------------------------------------ profiling
    def set_profiling(self, on: bool):
        check(_abi.load().fdtd_llg_set_profiling(self._h, 1 if on else 0), self._h)

    def read_profile(self, reset: bool = True) -> dict:
        pr = _abi.Profile()
        check(_abi.load().fdtd_llg_read_profile(self._h, C.byref(pr), 1 if reset else 0), self._h)
        kinds = ("step", "mag", "half")
        return {"cells": pr.cells, **{k: {"launches": pr.launches[q], "ms": pr.ms[q]} for q, k in enumerate(kinds)}}

    # ----------------------------------------------------------- cleanup
    def destroy(self):
        if self._root is self and self._h:
            _abi.load().fdtd_llg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
