"""fdtd_llg_e_push_noalloc: the E push for callers that cannot allocate
device memory (code living inside another framework's memory pool, or a
real-time loop where allocation is not allowed).  Its partial sums sit in a
fixed array inside the library instead of memory it allocates.

The test calls it through the C ABI on buffers the test owns, starting from a
non-zero E so that the ca E^n term of Eq. Ampere counts, and checks the new E
and its electric energy two ways: against the handle-based solver doing the
same update (fdtd_llg_step from the same stored E^n and H^{n+1/2}, written
with fdtd_llg_planes and read back with fdtd_llg_get_field), and against the
update written out in FP64 here.  Three calls in a row: the second continues
on the first call's output E in the same buffers with a new H and no energy
output, the third runs a larger lossy grid, so it reads partial-sum slots that
the earlier calls left behind and must overwrite."""
import ctypes as C

import numpy as np
import pytest

import paper_2510_22221_b300 as pkg
from paper_2510_22221_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 2e-5          # the parity tests' tolerance for one FP32 step
EPS0 = 1.0 / (4e-7 * np.pi * 299792458.0 ** 2)


def handle_push(nx, ny, nz, d, dt, eps_r, sigma, E, H):
    """E after one step of the handle-based solver whose stored state is
    E^n = E and H^{n+1/2} = H: the handle is first stepped once (into the
    state where H is stored half a step ahead of E), the planes are then
    overwritten with E and H, and its next step's E push is ca E + cb curl H."""
    mats = [W.material(eps_r=eps_r, sigma=sigma)]
    sim = pkg.FdtdLlg.create(nx, ny, nz, *d, dt=dt, probe_capacity=2)
    sim.set_materials(np.zeros((nz, ny, nx), np.uint8), [pkg.Material(**m) for m in mats], [0.0, 0.0, 0.0])
    sim.step(1)
    zero_walls = [np.zeros((nz, ny), np.float32), np.zeros((nz, nx), np.float32)]
    data = np.concatenate([a.ravel() for a in (*E, *H, *zero_walls)] + [np.zeros(3 * nz * ny * nx, np.float32)])
    sim.write_planes(0, nz, data)
    sim.step(1)
    out = [sim.get_field(n) for n in ("Ex", "Ey", "Ez")]
    sim.destroy()
    return out


def fp64_push(d, dt, eps_r, sigma, E, H):
    """Eq. Ampere, E^{n+1} = (sigma/2 + eps/dt)^{-1} [curl H - (sigma/2 - eps/dt) E^n],
    on the compact layout (Ex[k, j, i] at (i+1/2, j, k), H on the faces below
    and behind each edge), with every edge in a wall held at zero."""
    Ex, Ey, Ez = (np.asarray(a, np.float64) for a in E)
    Hx, Hy, Hz = (np.asarray(a, np.float64) for a in H)
    eps = EPS0 * eps_r
    den = sigma / 2 + eps / dt

    def back(a, axis):   # a - a shifted by one cell towards the low side (zero beyond)
        s = np.zeros_like(a)
        sl = [slice(None)] * 3
        sl[axis] = slice(1, None)
        sl2 = [slice(None)] * 3
        sl2[axis] = slice(None, -1)
        s[tuple(sl)] = a[tuple(sl2)]
        return a - s

    cx = back(Hz, 1) / d[1] - back(Hy, 0) / d[2]
    cy = back(Hx, 0) / d[2] - back(Hz, 2) / d[0]
    cz = back(Hy, 2) / d[0] - back(Hx, 1) / d[1]
    out = [(c - (sigma / 2 - eps / dt) * e) / den for c, e in ((cx, Ex), (cy, Ey), (cz, Ez))]
    out[0][:, 0, :] = 0.0
    out[0][0, :, :] = 0.0
    out[1][:, :, 0] = 0.0
    out[1][0, :, :] = 0.0
    out[2][:, :, 0] = 0.0
    out[2][:, 0, :] = 0.0
    return out


def noalloc_call(lib, Et, Ht, shape, d, dt, eps_r, sigma, with_energy):
    import torch

    nz, ny, nx = shape
    w = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    rc = lib.fdtd_llg_e_push_noalloc(*[C.c_void_p(t.data_ptr()) for t in Et], *[C.c_void_p(t.data_ptr()) for t in Ht],
                                     nx, ny, nz, *d, dt, eps_r, sigma,
                                     C.c_void_p(w.data_ptr()) if with_energy else None,
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.fdtd_llg_last_error(None)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in Et], float(w.item())


def check(got, refs):
    scale = max(float(np.abs(r).max()) for r in refs[0])
    assert scale > 0
    for ref in refs:
        for g, r in zip(got, ref):
            assert float(np.abs(g.astype(np.float64) - r).max()) <= TOL * scale


def test_noalloc_e_push_matches_step_on_calls_in_a_row():
    import torch

    lib = pkg.load_library()
    rng = np.random.default_rng(17)
    # call 1 and call 2 share one grid and its buffers; call 3 is larger and lossy
    (nx, ny, nz), d, eps_r, sigma = (37, 21, 19), (1.0e-6, 0.8e-6, 1.2e-6), 3.0, 0.0
    dt = 0.5 / (299792458.0 * np.sqrt(sum(1.0 / v ** 2 for v in d)))
    E0 = [rng.normal(size=(nz, ny, nx)).astype(np.float32) for _ in range(3)]
    H0 = [(300.0 * rng.normal(size=(nz, ny, nx))).astype(np.float32) for _ in range(3)]
    Et = [torch.from_numpy(e.copy()).cuda() for e in E0]
    Ht = [torch.from_numpy(h.copy()).cuda() for h in H0]
    got1, w1 = noalloc_call(lib, Et, Ht, (nz, ny, nx), d, dt, eps_r, sigma, True)
    ref1 = handle_push(nx, ny, nz, d, dt, eps_r, sigma, E0, H0)
    check(got1, [ref1, fp64_push(d, dt, eps_r, sigma, E0, H0)])
    w_ref = 0.5 * EPS0 * eps_r * d[0] * d[1] * d[2] * sum(float((r.astype(np.float64) ** 2).sum()) for r in ref1)
    assert abs(w1 - w_ref) <= TOL * w_ref, (w1, w_ref)

    # call 2: the same buffers, E as call 1 left it, a new H, no energy output
    H1 = [(300.0 * rng.normal(size=(nz, ny, nx))).astype(np.float32) for _ in range(3)]
    for t, h in zip(Ht, H1):
        t.copy_(torch.from_numpy(h))
    got2, w2 = noalloc_call(lib, Et, Ht, (nz, ny, nx), d, dt, eps_r, sigma, False)
    assert w2 == -1.0                     # w_e = NULL: nothing written
    check(got2, [handle_push(nx, ny, nz, d, dt, eps_r, sigma, got1, H1), fp64_push(d, dt, eps_r, sigma, got1, H1)])

    # call 3: a larger lossy grid (ca = (eps/dt - sigma/2) / (eps/dt + sigma/2) < 1)
    (nx, ny, nz), d, eps_r, sigma = (64, 33, 40), (0.5e-6, 0.5e-6, 0.7e-6), 2.0, 5e4
    dt = 0.5 / (299792458.0 * np.sqrt(sum(1.0 / v ** 2 for v in d)))
    E0 = [rng.normal(size=(nz, ny, nx)).astype(np.float32) for _ in range(3)]
    H0 = [(300.0 * rng.normal(size=(nz, ny, nx))).astype(np.float32) for _ in range(3)]
    Et = [torch.from_numpy(e.copy()).cuda() for e in E0]
    Ht = [torch.from_numpy(h.copy()).cuda() for h in H0]
    got3, w3 = noalloc_call(lib, Et, Ht, (nz, ny, nx), d, dt, eps_r, sigma, True)
    ref3 = handle_push(nx, ny, nz, d, dt, eps_r, sigma, E0, H0)
    check(got3, [ref3, fp64_push(d, dt, eps_r, sigma, E0, H0)])
    w_ref = 0.5 * EPS0 * eps_r * d[0] * d[1] * d[2] * sum(float((r.astype(np.float64) ** 2).sum()) for r in ref3)
    assert abs(w3 - w_ref) <= TOL * w_ref, (w3, w_ref)


def test_noalloc_rejects_grids_beyond_its_fixed_array():
    import torch

    lib = pkg.load_library()
    t = torch.zeros(8, dtype=torch.float32, device="cuda")
    p = C.c_void_p(t.data_ptr())
    rc = lib.fdtd_llg_e_push_noalloc(p, p, p, p, p, p, 2048, 2048, 2048, 1e-6, 1e-6, 1e-6, 1e-16, 1.0, 0.0, None, None)
    assert rc == -1
    assert b"limited to 65536" in lib.fdtd_llg_last_error(None)
