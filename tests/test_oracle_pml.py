"""Pins of the oracle's absorbing layers (reading R15: the convolutional PML of
Roden and Gedney with the complex-frequency-shifted stretch; the paper bounds
its device with PMLs but gives no formulation).

Each pin checks the oracle against something other than itself:
  * vanishing layers (sigma = 0, kappa = 1, alpha = 0) leave the scheme
    exactly the PEC-box scheme, bit for bit;
  * a matched layer reflects little: a line source's field at a probe agrees
    with the same run in a grid so large that its walls' echo arrives after
    the window, while a plain PEC wall at the layer's place echoes strongly;
  * the three 2-D orientations (plates normal to z, x, y) are rotations of
    one problem, so their probe series agree to rounding: a wrong index,
    sign or axis in any of the twelve memories breaks the agreement;
  * energy leaves a box lined with layers on every face;
  * an anisotropic problem rotated cyclically stays one problem, and a
    centred source's field stays mirror-symmetric across the low and high
    layers, to the last bit;
  * the reflection of a waveguide mode from a lined end equals, over a band
    of frequencies, the round-trip attenuation of the continuous stretch
    s = kappa + sigma / (alpha + j w eps0) graded as stated, which ties the
    layer's sigma and alpha profiles (their grading included) to the
    mathematics of the stretch.
"""
import numpy as np
import pytest

import oracle
from oracle import Material, OracleSim, Pml, Source

DX = 1e-3
F0 = 30e9


def _plates(orient, n, steps, pml=None, pad=0, d=10):
    """2-D run: axis `orient` is one cell thick (PEC plates), the line
    current flows along it at the centre, the probe sits 3 cells away."""
    N = [n + 2 * pad] * 3
    N[orient] = 1
    dt = oracle.courant_dt(DX, DX, DX, 0.99)
    c = [N[0] // 2, N[1] // 2, N[2] // 2]
    c[orient] = 0
    pr = list(c)
    pr[(orient + 1) % 3] += 3
    src = Source(comp=orient, ijk=tuple(c), J0=1.0, f0=F0, Tp=0.5 / F0, tpk=1.5 / F0)
    pm = None
    if pml is not None:
        layers = [d, d, d]
        layers[orient] = 0
        pm = Pml(n=tuple(layers), **pml)
    sim = OracleSim(*N, DX, DX, DX, dt, [Material()], np.zeros((N[2], N[1], N[0]), np.uint8), (0, 0, 0),
                    sources=[src], probes=[tuple(pr)], pml=pm)
    r = sim.run(steps)
    return r["probes"][:, 0, orient], r["energy"]


@pytest.fixture(scope="module")
def reference():
    # walls 120 cells from the source: their echo reaches the probe after
    # ~237 cells of travel, beyond the 300-step window (~170 cells)
    ref, _ = _plates(2, 40, 300, pad=100)
    return ref


@pytest.mark.parametrize("orient", [2, 0, 1])
def test_layers_absorb_what_a_wall_echoes(reference, orient):
    a, ea = _plates(orient, 40, 300, pml={})
    b, eb = _plates(orient, 40, 300)
    m = np.abs(reference).max()
    assert np.abs(a - reference).max() / m < 2e-3      # about -66 dB
    assert np.abs(b - reference).max() / m > 0.3       # the PEC wall's echo
    assert ea[-1] / ea.max() < 1e-5                    # the pulse has left
    assert eb[-1] / eb.max() > 0.9                     # a PEC box keeps it


def test_three_orientations_are_one_problem():
    runs = [_plates(o, 40, 200, pml=dict(kappa_max=3.0, alpha_max=0.2))[0] for o in (2, 0, 1)]
    m = np.abs(runs[0]).max()
    for r in runs[1:]:
        assert np.abs(r - runs[0]).max() / m < 1e-12


def test_stretched_and_shifted_layers_still_absorb(reference):
    a, _ = _plates(2, 40, 300, pml=dict(kappa_max=5.0, alpha_max=0.5))
    assert np.abs(a - reference).max() / np.abs(reference).max() < 1e-2


def _box(pml, nsteps=40, n=12):
    rng = np.random.default_rng(7)
    mats = [Material(), Material(eps_r=4.0, sigma=0.02), Material(Ms=1.4e5, alpha=0.01)]
    mid = np.zeros((n, n, n), np.uint8)
    mid[3:9, 2:10, 4:8] = 1
    mid[5:7, 5:7, 5:7] = 2
    dt = oracle.courant_dt(DX, DX, DX, 0.9)
    src = Source(comp=0, ijk=(6, 4, 4), J0=1e3, f0=F0)
    sim = OracleSim(n, n, n, DX, DX, DX, dt, mats, mid, (0.0, 0.0, 8e4), sources=[src],
                    probes=[(6, 6, 6), (2, 2, 2)], pml=pml)
    for nm in ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz"):
        a = getattr(sim, nm)
        sim.set_fields(**{nm: rng.standard_normal(a.shape)})
    r = sim.run(nsteps)
    return sim, r


def test_vanishing_layers_are_the_pec_box_exactly():
    s0, r0 = _box(None)
    s1, r1 = _box(Pml(n=(3, 4, 2), scale=0.0, kappa_max=1.0, alpha_max=0.0))
    for nm in ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz", "M"):
        assert np.array_equal(getattr(s0, nm), getattr(s1, nm)), nm
    assert np.array_equal(r0["probes"], r1["probes"])
    assert np.array_equal(r0["energy"], r1["energy"])
    assert all(not np.any(v) for v in s1.psi_blocks().values())


def test_layers_change_only_the_layers_at_first():
    """One step from the same state: with layers 2 cells deep, H and E change
    only within reach of the layers (the memory terms start from zero, so
    the first step differs from the PEC box only where sigma or kappa act)."""
    s0, _ = _box(None, nsteps=1)
    s1, _ = _box(Pml(n=(2, 2, 2), kappa_max=2.0), nsteps=1)
    dEx = np.abs(s0.Ex - s1.Ex)                        # (nz+1, ny+1, nx)
    assert dEx.max() > 0
    inner = dEx[4:-4, 4:-4, 4:-4]                      # two cells beyond the layers' reach
    assert inner.max() == 0


def test_energy_leaves_a_box_lined_on_every_face():
    n, d = 20, 5
    dt = oracle.courant_dt(DX, DX, DX, 0.99)
    # a one-period Gaussian (DC content exp(-2 pi^2), switched on at 1 % of its
    # peak): a point current with a net charge leaves a static dipole field
    # that no layer absorbs (here ~2e-5 of the peak energy)
    src = Source(comp=2, ijk=(10, 10, 10), J0=1.0, f0=F0)
    sims = [OracleSim(n, n, n, DX, DX, DX, dt, [Material()], np.zeros((n, n, n), np.uint8), (0, 0, 0),
                      sources=[src], pml=p) for p in (Pml(n=(d, d, d)), None)]
    ea, eb = (s.run(400)["energy"] for s in sims)
    assert ea[-1] / ea.max() < 1e-4
    assert eb[-1] / eb.max() > 0.1     # the PEC box keeps what the source left in it


def _plates_aniso(orient, steps=160):
    """Plates normal to axis `orient`; the in-plane axes a1 = orient+1 and
    a2 = orient+2 (mod 3) get different sizes (40, 48), spacings (1.0, 1.3
    mm) and layers (10, 6), the thin axis 0.8 mm: cyclic relabellings of one
    problem, which the curl equations map onto each other exactly."""
    a1, a2 = (orient + 1) % 3, (orient + 2) % 3
    N, D, L = [0] * 3, [0.0] * 3, [0] * 3
    N[orient], N[a1], N[a2] = 1, 40, 48
    D[orient], D[a1], D[a2] = 0.8e-3, 1.0e-3, 1.3e-3
    L[orient], L[a1], L[a2] = 0, 10, 6
    dt = oracle.courant_dt(*D, 0.95)
    c = [0, 0, 0]
    c[a1], c[a2] = 20, 24
    pr = list(c)
    pr[a1] += 3
    pr[a2] -= 2
    src = Source(comp=orient, ijk=tuple(c), J0=1.0, f0=F0, Tp=0.5 / F0, tpk=1.5 / F0)
    sim = OracleSim(*N, *D, dt, [Material()], np.zeros((N[2], N[1], N[0]), np.uint8), (0, 0, 0),
                    sources=[src], probes=[tuple(pr)],
                    pml=Pml(n=tuple(L), order=3.0, scale=1.3, kappa_max=2.5, alpha_max=0.3))
    return sim.run(steps)["probes"][:, 0, orient]


def test_anisotropic_problem_rotated_is_one_problem():
    """Distinct extents, spacings and layer counts per axis: a profile read
    on the wrong axis or graded with the wrong spacing breaks the equality."""
    runs = [_plates_aniso(o) for o in (2, 0, 1)]
    m = np.abs(runs[0]).max()
    assert m > 0
    for r in runs[1:]:
        assert np.abs(r - runs[0]).max() / m < 1e-12


def test_centred_line_field_is_mirror_symmetric():
    """A line current at the centre node of a square lined on both sides:
    the field must be the same at mirrored nodes, low layers against high
    ones, to the last bit (the depths rho of mirrored positions are equal
    exactly); a grading that treats the two sides differently breaks it."""
    n, d = 40, 10
    dt = oracle.courant_dt(DX, DX, DX, 0.99)
    src = Source(comp=2, ijk=(n // 2, n // 2, 0), J0=1.0, f0=F0, Tp=0.5 / F0, tpk=1.5 / F0)
    sim = OracleSim(n, n, 1, DX, DX, DX, dt, [Material()], np.zeros((1, n, n), np.uint8), (0, 0, 0),
                    sources=[src], pml=Pml(n=(d, d, 0), kappa_max=2.0, alpha_max=0.2))
    sim.run(150)                              # the pulse has crossed the layers and come back
    ez = sim.Ez[0]                            # (ny+1, nx+1) nodes
    m = np.abs(ez).max()
    assert np.abs(ez[:, n // 2 + 15]).max() > 1e-6 * m     # field inside the high x layers
    assert np.array_equal(ez, ez[:, ::-1])
    assert np.array_equal(ez, ez[::-1, :])
    assert np.array_equal(ez, ez.T)


def test_cfs_layer_reflection_equals_the_stretched_coordinate_closed_form():
    """A rectangular waveguide along x (PEC walls; 40 cells of 1 mm across y,
    one cell in z) carries the TE10 mode, driven by z-currents across the
    guide weighted sin(pi y / b) (the discrete mode, so no other mode is
    excited), with a 15 GHz pulse.  Layers of d = 10 cells line both x ends
    (m = 3, sigma scale 0.3, kappa 1, alpha_max 5 S/m).  In a stretched
    coordinate the mode goes as exp(-j k_x integral s dx), k_x = sqrt(w^2/c^2 -
    (pi/b)^2); with s = kappa + sigma / (alpha + j w eps0) its amplitude falls
    by exp(-k_x integral sigma w eps0 / (alpha^2 + w^2 eps0^2) dx) each way,
    and the PEC wall behind the layer returns it, so the reflection is

        R(w) = exp(-2 k_x integral_0^d sigma w eps0 / (alpha^2 + w^2 eps0^2) dx)

    with sigma = sigma_max rho^m and alpha = alpha_max (1 - rho) at depth rho.
    The reflected wave is the probe series of the lined guide minus that of a
    guide long enough that its far end's echo arrives after the window (the
    near end and the source sit identically in both); |R| is the ratio of the
    two spectra.  The discrete layers absorb about 6 % more than the
    continuous stretch (in ln R; 3.7 % at half the time step: the memory
    recursion's discretisation), the same at every frequency; the bound is
    12 % of ln R.  The reversed grading alpha = alpha_max rho would give ln R
    about 18 times smaller (R 0.67-0.90 against 0.05-0.15 here)."""
    c, eps0 = oracle.c0(), oracle.eps0()
    eta0 = oracle.mu0() * c
    d, ny, L, m, scale, amax, f0 = 1e-3, 40, 10, 3.0, 0.3, 5.0, 15e9
    xs, xp, steps = 300, 550, 2700
    dt = oracle.courant_dt(d, d, d, 0.5)
    src = [Source(comp=2, ijk=(xs, j, 0), J0=float(np.sin(np.pi * j / ny)), f0=f0) for j in range(1, ny)]
    threads = oracle.set_threads(0)
    try:
        series = []
        for nx in (610, 1000):
            sim = OracleSim(nx, ny, 1, d, d, d, dt, [Material()], np.zeros((1, ny, nx), np.uint8), (0, 0, 0),
                            sources=src, probes=[(xp, ny // 2, 0)],
                            pml=Pml(n=(L, 0, 0), order=m, scale=scale, kappa_max=1.0, alpha_max=amax))
            series.append(sim.run(steps)["probes"][:, 0, 2])
    finally:
        oracle.set_threads(1)
    assert threads >= 1
    lined, long_ = series
    # the windows hold the whole reflected pulse and nothing of a second echo
    assert np.abs(long_[-200:]).max() < 2e-3 * np.abs(long_).max()
    freqs = np.linspace(10e9, 20e9, 11)
    ph = np.exp(-2j * np.pi * np.outer(freqs, np.arange(steps) * dt))
    R_meas = np.abs(ph @ (lined - long_)) / np.abs(ph @ long_)
    w = 2 * np.pi * freqs
    kx = np.sqrt((w / c) ** 2 - (np.pi / (ny * d)) ** 2)
    rho = (np.arange(4000) + 0.5) / 4000
    sig = scale * 0.8 * (m + 1) / (eta0 * d) * rho ** m

    def closed_form(alpha):
        integral = np.array([np.mean(sig * wi * eps0 / (alpha ** 2 + (wi * eps0) ** 2)) * L * d for wi in w])
        return np.exp(-2 * kx * integral)

    R_th = closed_form(amax * (1 - rho))
    ratio = np.log(R_meas) / np.log(R_th)
    assert np.all(np.abs(ratio - 1) < 0.12), ratio
    assert np.ptp(ratio) < 0.02, ratio          # the same excess at every frequency
    R_rev = closed_form(amax * rho)
    assert np.all(np.log(R_rev) / np.log(R_th) < 0.2)
