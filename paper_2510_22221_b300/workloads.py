"""Seeded synthetic workloads (geometry, materials, sources, probes).

This module only lays out inputs; it holds none of the method's arithmetic
(no time step, no field update).  Both the CUDA path and the FP64 oracle are
driven from the same ``Workload`` objects.  The shapes follow the paper's
workload family (section "Modeling Setup": a strip resonator on a high-eps
substrate loaded by a thin ferromagnetic film, excited by a modulated
Gaussian) at the sizes given for each configuration; the paper's CPW device
with PML and its dataset are not reproduced.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

MU0 = 4e-7 * np.pi   # only to express a bias given in tesla as A/m


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    courant: float                       # dt = courant x 3-D Courant limit
    steps: int
    materials: list                      # dicts: eps_r, sigma, Ms, alpha, gamma, pec
    mat_id: np.ndarray                   # uint8 (nz, ny, nx)
    hbias: np.ndarray                    # A/m
    sources: list = field(default_factory=list)   # dicts: comp, i, j, k, J0, f0, Tp, tpk
    probes: list = field(default_factory=list)    # (i, j, k)
    eps_design: np.ndarray | None = None # (nk, nj, ni) eps_r over design_box
    design_box: tuple | None = None      # (i0, j0, k0, ni, nj, nk)
    note: str = ""
    pml: dict | None = None              # absorbing layers: layers (x, y, z), order, scale, kappa_max, alpha_max

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def eps_r_cell(self) -> np.ndarray:
        """Per-cell eps_r (table values with the design box overridden)."""
        eps = np.array([m["eps_r"] for m in self.materials])[self.mat_id]
        if self.eps_design is not None:
            i0, j0, k0, ni, nj, nk = self.design_box
            eps[k0:k0 + nk, j0:j0 + nj, i0:i0 + ni] = self.eps_design
        return eps


def material(eps_r=1.0, sigma=0.0, Ms=0.0, alpha=0.0, gamma=1.76e11, pec=False) -> dict:
    return dict(eps_r=eps_r, sigma=sigma, Ms=Ms, alpha=alpha, gamma=gamma, pec=pec)


YIG = dict(Ms=1.4e5, alpha=1e-3, gamma=1.76e11)


def cavity_block(n=32, steps=2000) -> Workload:
    """32^3 PEC box, dx = 1 um, vacuum; YIG block of 8x8x2 cells at the centre
    (cells 12-19, 12-19, 15-16), M along a 0.1 T bias on z; x-directed point
    current at the edge (16.5, 16, 14) next to the block, 5 GHz modulated
    Gaussian; one probe in the cell (20, 16, 15) next to the block."""
    mats = [material(), material(eps_r=1.0, **YIG)]
    mid = np.zeros((n, n, n), dtype=np.uint8)
    c = n // 2
    mid[c - 1:c + 1, c - 4:c + 4, c - 4:c + 4] = 1
    src = [dict(comp=0, i=c, j=c, k=c - 2, J0=1.0, f0=5e9, Tp=0.0, tpk=0.0)]
    return Workload(f"cavity_block_{n}", n, n, n, 1e-6, 1e-6, 1e-6, 0.5, steps, mats, mid,
                    np.array([0.0, 0.0, 0.1 / MU0]), src, [(c + 4, c, c - 1)],
                    note="PEC box, vacuum, 8x8x2 YIG block, 0.1 T on z, 5 GHz x-current")


def strip_resonator(nx=256, ny=256, nz=128, steps=20000, strips=1, film=(40, 8, 4), alpha=1e-3, J0=1.0,
                    bias_tesla=20.9, name=None) -> Workload:
    """dx = 0.5 um PEC box; substrate eps_r = 12 fills the lower half z < nz/2;
    PEC strip(s) 4 x 200 cells (x, y), one cell thick, on the substrate at
    z = nz/2, centred in y and spread evenly in x; a YIG film of film = (x, y, z)
    cells under each strip, replacing substrate at z in [nz/2 - 4, nz/2).
    Bias along y (the strip's long axis, as the paper biases along the line);
    bias_tesla is a fixed stand-in for the value that tunes the film's Kittel
    frequency to the strip's half-wave resonance (~0.6 THz for a 100 um strip
    in eps_eff ~ 6.5).  Source: x-current in the gap beside strip 0 near its
    end; probes beside and inside the film of strip 0."""
    mats = [material(), material(eps_r=12.0), material(pec=True), material(eps_r=12.0, Ms=YIG["Ms"],
                                                                           alpha=alpha, gamma=YIG["gamma"])]
    mid = np.zeros((nz, ny, nx), dtype=np.uint8)
    zs = nz // 2
    mid[:zs] = 1
    fx, fy, fz = film
    centres = [int(round((q + 0.5) * nx / strips)) for q in range(strips)]
    y0 = (ny - 200) // 2
    for cx in centres:
        mid[zs, y0:y0 + 200, cx - 2:cx + 2] = 2
        mid[zs - fz:zs, ny // 2 - fy // 2:ny // 2 - fy // 2 + fy, cx - fx // 2:cx - fx // 2 + fx] = 3
    cx = centres[0]
    src = [dict(comp=0, i=cx + 3, j=y0 + 10, k=zs + 1, J0=J0, f0=6e11, Tp=0.0, tpk=0.0)]
    probes = [(cx - fx // 2 - 1, ny // 2, zs - 2), (cx, ny // 2, zs - 2)]
    return Workload(name or f"strip_resonator_{nx}x{ny}x{nz}", nx, ny, nz, 0.5e-6, 0.5e-6, 0.5e-6, 0.5, steps,
                    mats, mid, np.array([0.0, bias_tesla / MU0, 0.0]), src, probes,
                    note=f"{strips} PEC strip(s) 4x200 on eps_r=12 substrate, YIG film {fx}x{fy}x{fz} under each, "
                         f"bias {bias_tesla} T along y")


def multi_strip(steps=50000) -> Workload:
    """512 x 512 x 256, eight strips each loaded by a 64 x 12 x 4 YIG film,
    alpha = 1e-4, drive amplitude 1e6 times the linear configurations'.  Each
    film lies along its strip: 64 cells in y, 12 across in x, 4 thick; the
    strips are 64 cells apart in x, so the films stay separate magnetic
    regions (64 cells across would make the eight one connected 512-cell
    band, beyond one region's size)."""
    return strip_resonator(512, 512, 256, steps, strips=8, film=(12, 64, 4), alpha=1e-4, J0=1e6,
                           name="multi_strip_512x512x256")


def bias_sweep(n_inst=64, steps=10000, seed=0, L=7.57e-2) -> list:
    """Uneven cubes n_i ~ U{48..96} (seed), fixed physical side L = 7.57 cm
    (TE101 ~ 2.8 GHz), dx_i = L/n_i; vacuum; a YIG block of sides ~ U{4..16}
    (seed+1) centred in x, y and resting on the z = 0 wall; bias along z swept
    linearly over 0.05..0.15 T; x-current at the box centre, 2.8 GHz; one probe
    beside the block."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(48, 97, size=n_inst)
    rng2 = np.random.default_rng(seed + 1)
    mag = rng2.integers(4, 17, size=(n_inst, 3))
    out = []
    for q in range(n_inst):
        n = int(sides[q])
        mx, my, mz = (int(v) for v in mag[q])
        mats = [material(), material(eps_r=1.0, **YIG)]
        mid = np.zeros((n, n, n), dtype=np.uint8)
        x0, y0 = n // 2 - mx // 2, n // 2 - my // 2
        mid[0:mz, y0:y0 + my, x0:x0 + mx] = 1
        b = 0.05 + 0.1 * q / max(n_inst - 1, 1)
        d = L / n
        src = [dict(comp=0, i=n // 2, j=n // 2, k=n // 2, J0=1.0, f0=2.8e9, Tp=0.0, tpk=0.0)]
        probes = [(min(x0 + mx, n - 1), n // 2, 1)]
        out.append(Workload(f"sweep_{q}_n{n}", n, n, n, d, d, d, 0.5, steps, mats, mid,
                            np.array([0.0, 0.0, b / MU0]), src, probes,
                            note=f"cube n={n}, magnet {mx}x{my}x{mz}, bias {b:.4f} T"))
    return out


def anticrossing_sweep(n_inst=5, b_lo=0.0375, b_hi=0.06, steps=16000, nx=24, ny=16, nz=5, d=3.15e-3,
                       mag=(4, 4, 2), design=None, seed=3) -> list:
    """A bias sweep through one magnon-photon anti-crossing at a size the FP64
    oracle runs in seconds: a flat PEC box (nx, ny, nz cells of side d: 7.6 x
    5.0 x 1.6 cm) whose only mode near 3.6 GHz is TM110 (E along z, H in the
    x-y plane, largest at the y = 0 wall); a YIG block mx x my x mz against
    that wall, centred in x and z; bias along z from b_lo to b_hi (T), over
    which the block's uniform precession mode crosses TM110 (the splitting is
    smallest near 0.05 T for the default block); z-current at the box centre,
    3.7 GHz pulse; probe at the centre (E_z).  Higher magnetostatic modes of
    the block cross the cavity mode above ~0.06 T."""
    out = []
    mx, my, mz = mag
    for q in range(n_inst):
        mats = [material(), material(eps_r=1.0, **YIG)]
        mid = np.zeros((nz, ny, nx), dtype=np.uint8)
        x0, z0 = nx // 2 - mx // 2, nz // 2 - mz // 2
        mid[z0:z0 + mz, 0:my, x0:x0 + mx] = 1
        b = b_lo + (b_hi - b_lo) * q / max(n_inst - 1, 1)
        src = [dict(comp=2, i=nx // 2, j=ny // 2, k=nz // 2, J0=1.0, f0=3.7e9, Tp=0.0, tpk=0.0)]
        probes = [(nx // 2, ny // 2, nz // 2)]
        eps, box = None, None
        if design is not None:   # a dielectric design box between the source and the magnet
            ddx, ddy, ddz = design
            box = (nx // 2 - ddx // 2, my + 1, nz // 2 - ddz // 2, ddx, ddy, ddz)
            eps = np.random.default_rng(seed).uniform(1.0, 4.0, size=(ddz, ddy, ddx))
        out.append(Workload(f"anticross_{q}", nx, ny, nz, d, d, d, 0.5, steps, mats, mid,
                            np.array([0.0, 0.0, b / MU0]), src, probes, eps_design=eps, design_box=box,
                            note=f"flat box {nx}x{ny}x{nz}, magnet {mx}x{my}x{mz} on the y=0 wall, bias {b:.4f} T"))
    return out


def quasi1d_film(h_oe=(1700.0, 1800.0, 1900.0), nx=20160, ny=32, thickness=0.7e-6, width=0.32,
                 steps=680000) -> list:
    """The supplement's film in a closed cavity that keeps its fields 1-D
    (Supplementary Information, Table S1 materials; one instance per bias
    field h_oe, in oersted).  A parallel-plate resonator: nx cells of the
    film's thickness along x (1.41 cm, PEC ends), ny cells across y (width
    0.32 m between PEC walls, so that the field's transverse sine varies
    ~10^4 times more slowly than the film is thick), one cell along z;
    its fundamental mode (E along z, H in the x-y plane) lies near
    10.63 GHz.  A film one cell thick spans the cross-section at
    i = nx // 8 (Ms 9.7e5 A/m, gamma' = mu0 gamma = 2.23e5, alpha 0.003,
    eps_r 1, sigma 1e-3 S/m); the cavity is vacuum with sigma 1e-3 S/m.
    Bias along z (in the film's plane); the film's uniform precession
    crosses the cavity mode near 1800 Oe.  No source: the run starts from
    a tilted film.  Probe at the film's centre cell."""
    oe = 1e3 / (4 * np.pi)
    dy = width / ny
    i_f = nx // 8
    out = []
    for h in h_oe:
        mats = [material(sigma=1e-3), material(eps_r=1.0, sigma=1e-3, Ms=9.7e5, alpha=0.003, gamma=2.23e5 / MU0)]
        mid = np.zeros((1, ny, nx), dtype=np.uint8)
        mid[0, :, i_f] = 1
        out.append(Workload(f"quasi1d_{h:.0f}oe", nx, ny, 1, thickness, dy, dy, 0.95, steps, mats, mid,
                            np.array([0.0, 0.0, h * oe]), [], [(i_f, ny // 2, 0)],
                            note=f"quasi-1-D resonator {nx}x{ny}x1, film at i = {i_f}, bias {h:.0f} Oe along z"))
    return out


def adjoint_design(nx=128, ny=128, nz=64, steps=4000, seed=2, design=(32, 32, 4), block=(16, 16, 4)) -> Workload:
    """dx = 0.5 um PEC box, vacuum; design region design = (x, y, z) cells with
    eps_r ~ U[1, 12] (seed) between the source and the probe; a YIG block of
    block cells beside it; x-current source and probe on the x axis through the
    centre."""
    rng = np.random.default_rng(seed)
    mats = [material(), material(eps_r=1.0, **YIG)]
    mid = np.zeros((nz, ny, nx), dtype=np.uint8)
    cx, cy, cz = nx // 2, ny // 2, nz // 2
    bx, by, bz = block
    mid[cz - bz // 2:cz - bz // 2 + bz, cy - by // 2:cy - by // 2 + by, cx + 8:cx + 8 + bx] = 1
    dx_, dy_, dz_ = design
    box = (cx - dx_ // 2 - 8, cy - dy_ // 2, cz - dz_ // 2, dx_, dy_, dz_)
    eps = rng.uniform(1.0, 12.0, size=(dz_, dy_, dx_))
    src = [dict(comp=0, i=box[0] - 6, j=cy, k=cz, J0=1.0, f0=2e12, Tp=0.0, tpk=0.0)]
    probes = [(cx + 8 + bx + 4, cy, cz)]
    return Workload(f"adjoint_design_{nx}x{ny}x{nz}", nx, ny, nz, 0.5e-6, 0.5e-6, 0.5e-6, 0.5, steps, mats, mid,
                    np.array([0.0, 0.0, 0.1 / MU0]), src, probes, eps_design=eps, design_box=box,
                    note=f"design {dx_}x{dy_}x{dz_} eps_r~U[1,12], YIG {bx}x{by}x{bz}")


def adjoint_small(n=24, steps=400, seed=2, design=(8, 8, 2), block=(4, 4, 2), f0=20e12) -> Workload:
    """The adjoint case at a size the FP64 oracle differentiates in seconds:
    an n^3 PEC box of 0.5 um cells, vacuum; a design region of design cells
    with eps_r ~ U[1, 12] (seed) between an x-current source and an E probe on
    the x axis through the centre, a YIG block past the design region (0.1 T
    on z).  f0 = 20 THz puts several wavelengths between source and probe."""
    rng = np.random.default_rng(seed)
    mats = [material(), material(eps_r=1.0, **YIG)]
    mid = np.zeros((n, n, n), dtype=np.uint8)
    c = n // 2
    dx_, dy_, dz_ = design
    bx, by, bz = block
    x_d = n // 6
    box = (x_d, c - dy_ // 2, c - dz_ // 2, dx_, dy_, dz_)
    x_m = x_d + dx_ + 2
    mid[c - bz // 2:c - bz // 2 + bz, c - by // 2:c - by // 2 + by, x_m:x_m + bx] = 1
    eps = rng.uniform(1.0, 12.0, size=(dz_, dy_, dx_))
    src = [dict(comp=0, i=max(x_d - 2, 1), j=c, k=c, J0=1.0, f0=f0, Tp=0.0, tpk=0.0)]
    probes = [(min(x_m + bx + 2, n - 2), c, c)]
    return Workload(f"adjoint_small_{n}", n, n, n, 0.5e-6, 0.5e-6, 0.5e-6, 0.5, steps, mats, mid,
                    np.array([0.0, 0.0, 0.1 / MU0]), src, probes, eps_design=eps, design_box=box,
                    note=f"{n}^3, design {dx_}x{dy_}x{dz_} eps_r~U[1,12], YIG {bx}x{by}x{bz}")


def random_small(seed, nx=13, ny=11, nz=9, steps=40, magnets=True, sigma=0.0, design=False) -> Workload:
    """Small ragged grid with every feature: dielectric, lossy dielectric,
    PEC cells, two magnetic materials in several regions (one touching the
    far x wall), a design box, two sources and three probes; bias of 2 T in a
    random direction.  Drive amplitudes ~1e6 A/m^2 keep the fields far above
    FP64 rounding of the static magnetisation (~1e-16 Ms)."""
    rng = np.random.default_rng(seed)
    mats = [material(), material(eps_r=4.0, sigma=sigma), material(pec=True),
            material(eps_r=2.0, Ms=1.4e5, alpha=0.01, gamma=1.76e11),
            material(eps_r=1.0, Ms=0.9e5, alpha=0.05, gamma=1.5e11)]
    mid = np.zeros((nz, ny, nx), dtype=np.uint8)
    mid[: nz // 3] = 1
    mid[nz // 2, 2:5, 3] = 2
    if magnets:
        mid[2:5, 3:6, 4:8] = 3
        mid[5:7, 6:9, nx - 3:nx] = 4                 # touches the far x wall
        mid[nz - 2, 1, 1] = 3                        # a single-cell region
    box = None
    eps = None
    if design:
        box = (6, 1, 4, 3, 2, 2)
        eps = rng.uniform(1.0, 12.0, size=(2, 2, 3))
    src = [dict(comp=0, i=5, j=5, k=4, J0=3e6, f0=4e12, Tp=2e-13, tpk=4e-13),
           dict(comp=2, i=8, j=3, k=6, J0=-2e6, f0=7e12, Tp=1.5e-13, tpk=3e-13)]
    probes = [(6, 4, 3), (nx - 2, 7, 5), (0, 0, 0)]
    h0 = rng.normal(size=3)
    h0 = h0 / np.linalg.norm(h0) * (2.0 / MU0)
    return Workload(f"random_small_{seed}", nx, ny, nz, 1e-6, 1.3e-6, 0.8e-6, 0.6, steps, mats, mid, h0, src, probes,
                    eps_design=eps, design_box=box, note="feature coverage")


def pml_small(seed, nx=30, ny=26, nz=22, steps=60, layers=(6, 5, 4), kappa_max=1.0, alpha_max=0.0) -> Workload:
    """Ragged grid bounded by absorbing layers: a lossy substrate and a PEC
    strip that run into the layers (a line ended by them), a magnetic block
    in the middle clear of the layers, two sources (one inside the layers),
    probes inside the layers, beside the block and in the far corner; bias of
    2 T in a random direction."""
    rng = np.random.default_rng(seed)
    mats = [material(), material(eps_r=4.0, sigma=2e3), material(pec=True),
            material(eps_r=2.0, Ms=1.4e5, alpha=0.01, gamma=1.76e11)]
    mid = np.zeros((nz, ny, nx), dtype=np.uint8)
    mid[: nz // 3] = 1
    mid[nz // 3, ny // 2 - 1:ny // 2 + 1, :] = 2
    mid[nz // 2 - 1:nz // 2 + 1, ny // 2 - 2:ny // 2 + 2, nx // 2 - 3:nx // 2 + 3] = 3
    src = [dict(comp=1, i=nx // 2 - 5, j=ny // 2 + 3, k=nz // 2, J0=3e6, f0=4e12, Tp=2e-13, tpk=4e-13),
           dict(comp=2, i=2, j=ny // 2 + 4, k=nz // 2 + 1, J0=-2e6, f0=7e12, Tp=1.5e-13, tpk=3e-13)]
    probes = [(nx // 2 + 5, ny // 2, nz // 2), (2, 3, 2), (nx - 2, ny - 2, nz - 2)]
    h0 = rng.normal(size=3)
    h0 = h0 / np.linalg.norm(h0) * (2.0 / MU0)
    return Workload(f"pml_small_{seed}", nx, ny, nz, 1e-6, 1.3e-6, 0.8e-6, 0.6, steps, mats, mid, h0, src, probes,
                    note="absorbing layers, lossy substrate and strip running into them, magnet clear of them",
                    pml=dict(layers=tuple(layers), order=3.0, scale=1.0, kappa_max=kappa_max, alpha_max=alpha_max))


def strip_resonator_pml(nx=256, ny=256, nz=128, steps=20000, layers=(10, 10, 8)) -> Workload:
    """The strip resonator with absorbing layers lining every face instead of
    bare PEC walls (the paper bounds its device by PMLs)."""
    w = strip_resonator(nx, ny, nz, steps, name=f"strip_resonator_pml_{nx}x{ny}x{nz}")
    w.pml = dict(layers=tuple(layers), order=3.0, scale=1.0, kappa_max=1.0, alpha_max=0.0)
    w.note += f", absorbing layers {layers}"
    return w


def cpw_device(steps=1000, layers=(10, 10, 10), h0_oe=2000.0, metal="sigma", film=True, split=False) -> Workload:
    """The paper's CPW resonator (section "Modeling Setup") on its own
    120 x 250 x 1000 grid of 5 x 19 x 1 um cells (dt = 2.94e-15 s at CFL 0.9):
    silicon substrate (eps_r 11.4) 500 um thick (z < 500), a 2 um metal
    layer on it (z 500-501: ground planes 250 um wide at both x edges,
    centre line 50 um wide with 25 um gaps, 198 cells = 3.76 mm long, gaps of
    10 cells = 190 um to feeding patches of 16 cells = 304 um at both y ends),
    a permalloy film (4 pi Ms = 1.2e4 G, alpha 0.003) 5 um thick and 30 um
    wide on the centre line, 148 cells = 2.81 mm long, in one piece (split=True
    cuts it by one non-magnetic cell at its middle, the variant that fitted
    one magnet CTA per half);
    bias H0 along y; absorbing layers on all six faces (the substrate, the
    grounds and the feeding patches run into them).  Metal: sigma = 1e11 S/m
    ("sigma") or PEC ("pec").  The voltage port is replaced by an x-directed
    current in the gap beside the first feeding patch, f0 = 16 GHz,
    Tp = 0.0625 ns; probes beside the film's middle and at the line's end.
    film=False leaves the film out (the bare resonator)."""
    nx, ny, nz = 120, 250, 1000
    dx, dy, dz = 5e-6, 19e-6, 1e-6
    metal_m = material(pec=True) if metal == "pec" else material(eps_r=1.0, sigma=1e11)
    py_ms = 1.2e4 / (4 * np.pi) * 1e3          # 4 pi Ms in gauss -> Ms in A/m
    mats = [material(), material(eps_r=11.4), metal_m, material(eps_r=1.0, Ms=py_ms, alpha=3e-3, gamma=1.76e11)]
    mid = np.zeros((nz, ny, nx), dtype=np.uint8)
    zs = 500
    mid[:zs] = 1
    m = mid[zs:zs + 2]                           # the metal layer (view)
    m[:, :, :50] = 2                             # ground planes
    m[:, :, 70:] = 2
    y0 = (ny - 198) // 2                         # centre line y 26..223
    m[:, y0:y0 + 198, 55:65] = 2
    m[:, :16, 55:65] = 2                         # feeding patches
    m[:, ny - 16:, 55:65] = 2
    fy0 = ny // 2 - 74                           # film y 51..198, split at 125
    if film:
        mid[zs + 2:zs + 7, fy0:fy0 + 148, 57:63] = 3
        if split:
            mid[zs + 2:zs + 7, ny // 2, 57:63] = 0
    src = [dict(comp=0, i=52, j=13, k=zs, J0=1.0, f0=16e9, Tp=0.0625e-9, tpk=0.0)]
    probes = [(56, ny // 2 + 30, zs + 8), (60, y0 + 2, zs + 2)]
    h0 = h0_oe * 1e3 / (4 * np.pi)              # oersted -> A/m
    return Workload(f"cpw_device_{nx}x{ny}x{nz}", nx, ny, nz, dx, dy, dz, 0.9, steps, mats, mid,
                    np.array([0.0, h0, 0.0]), src, probes,
                    note=f"paper's CPW resonator, {('split ' if split else '') + 'permalloy film on the centre line' if film else 'no film'}, H0 {h0_oe} Oe along y, "
                         f"absorbing layers {layers}, metal {metal}",
                    pml=dict(layers=tuple(layers), order=3.0, scale=1.0, kappa_max=1.0, alpha_max=0.0))


CONFIGS = {
    "cavity_block_32": cavity_block,
    "strip_resonator_256x256x128": strip_resonator,
    "bias_sweep_64": bias_sweep,
    "adjoint_design_128x128x64": adjoint_design,
    "multi_strip_512x512x256": multi_strip,
}
