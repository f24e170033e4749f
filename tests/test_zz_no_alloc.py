"""fdtd_llg_e_push_noalloc: the E push for callers that cannot allocate
device memory (code living inside another framework's memory pool, or a
real-time loop where allocation is not allowed).  Its partial sums sit in a
fixed array inside the library instead of memory it allocates.

The test calls it through the C ABI on buffers the test owns and checks the
new E field and its electric energy against the handle-based solver doing the
same update (fdtd_llg_step on a uniform medium, read back with
fdtd_llg_get_field), on two calls in a row of different sizes so that the
second call runs on the array the first one left behind."""
import ctypes as C

import numpy as np
import pytest

import paper_2510_22221_b300 as pkg
from paper_2510_22221_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 2e-5          # the parity tests' tolerance for one FP32 step
EPS0 = 1.0 / (4e-7 * np.pi * 299792458.0 ** 2)


def reference_push(nx, ny, nz, d, dt, eps_r, sigma, H):
    """E after one step of the handle-based solver from E = 0 and the given H
    (its first half-push leaves H unchanged because curl E = 0)."""
    mats = [W.material(eps_r=eps_r, sigma=sigma)]
    sim = pkg.FdtdLlg.create(nx, ny, nz, *d, dt=dt, probe_capacity=2)
    sim.set_materials(np.zeros((nz, ny, nx), np.uint8), [pkg.Material(**m) for m in mats], [0.0, 0.0, 0.0])
    for name, v in zip(("Hx", "Hy", "Hz"), H):
        sim.set_field(name, v)
    sim.step(1)
    E = [sim.get_field(n) for n in ("Ex", "Ey", "Ez")]
    sim.destroy()
    return E


def noalloc_push(lib, nx, ny, nz, d, dt, eps_r, sigma, H):
    import torch

    Et = [torch.zeros((nz, ny, nx), dtype=torch.float32, device="cuda") for _ in range(3)]
    Ht = [torch.from_numpy(np.ascontiguousarray(h)).cuda() for h in H]
    w = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    rc = lib.fdtd_llg_e_push_noalloc(*[C.c_void_p(t.data_ptr()) for t in Et], *[C.c_void_p(t.data_ptr()) for t in Ht],
                                     nx, ny, nz, *d, dt, eps_r, sigma, C.c_void_p(w.data_ptr()),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.fdtd_llg_last_error(None)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in Et], float(w.item())


def test_noalloc_e_push_matches_step_on_two_calls():
    lib = pkg.load_library()
    rng = np.random.default_rng(17)
    cases = [((37, 21, 19), (1.0e-6, 0.8e-6, 1.2e-6), 3.0, 0.0),
             ((64, 33, 40), (0.5e-6, 0.5e-6, 0.7e-6), 2.0, 5e3)]
    for (nx, ny, nz), d, eps_r, sigma in cases:
        dt = 0.5 / (299792458.0 * np.sqrt(sum(1.0 / v ** 2 for v in d)))
        H = [rng.normal(size=(nz, ny, nx)).astype(np.float32) for _ in range(3)]
        ref = reference_push(nx, ny, nz, d, dt, eps_r, sigma, H)
        got, w_e = noalloc_push(lib, nx, ny, nz, d, dt, eps_r, sigma, H)
        scale = max(float(np.abs(r).max()) for r in ref)
        assert scale > 0
        for g, r in zip(got, ref):
            assert float(np.abs(g.astype(np.float64) - r).max()) <= TOL * scale
        w_ref = 0.5 * EPS0 * eps_r * d[0] * d[1] * d[2] * sum(float((r.astype(np.float64) ** 2).sum()) for r in ref)
        assert abs(w_e - w_ref) <= TOL * w_ref, (w_e, w_ref)


def test_noalloc_rejects_grids_beyond_its_fixed_array():
    import torch

    lib = pkg.load_library()
    t = torch.zeros(8, dtype=torch.float32, device="cuda")
    p = C.c_void_p(t.data_ptr())
    rc = lib.fdtd_llg_e_push_noalloc(p, p, p, p, p, p, 2048, 2048, 2048, 1e-6, 1e-6, 1e-6, 1e-16, 1.0, 0.0, None, None)
    assert rc == -1
    assert b"limited to 65536" in lib.fdtd_llg_last_error(None)
