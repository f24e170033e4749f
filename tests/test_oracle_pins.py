"""Pins for the FP64 oracle against things other than itself: values the paper
prints, closed forms, invariants and a brute-force operator restatement
(arxiv 2510.22221, section "Numerical Model")."""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import Material, OracleSim, Source
from oracle import closed_forms as cf
from oracle.operators import YeeGeometry, maxwell_step_matrices


def _read_rows(path):
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _sig_round(x, digits):
    if x == 0:
        return 0.0
    return round(x, -int(math.floor(math.log10(abs(x)))) + (digits - 1))


# ----------------------------------------------------------- printed values
def test_courant_step_matches_printed(golden_dir):
    (row,) = _read_rows(os.path.join(golden_dir, "courant_modeling_setup.txt"))
    dx, dy, dz, cfl, dt_printed, digits = map(float, row)
    dt = oracle.courant_dt(dx, dy, dz, cfl)
    assert _sig_round(dt, int(digits)) == pytest.approx(dt_printed, rel=1e-12)
    assert dt == pytest.approx(cf.courant_dt(dx, dy, dz, cfl), rel=1e-15)


def test_kittel_formula_matches_printed(golden_dir):
    for kind, H0, Ms, gam, f_printed, digits in _read_rows(os.path.join(golden_dir, "kittel_printed.txt")):
        H0, Ms, gam, f_printed, digits = float(H0), float(Ms), float(gam), float(f_printed), int(digits)
        if kind == "cgs":
            f = cf.kittel_cgs_hz(H0, Ms, gam)
        else:
            f = cf.kittel_si_hz(H0 * cf.OE_TO_A_PER_M, Ms, gam)
        assert _sig_round(f, digits) == pytest.approx(f_printed, rel=1e-12), (kind, f)


def test_oracle_constants():
    assert oracle.mu0() == pytest.approx(4e-7 * math.pi, rel=1e-15)
    assert oracle.c0() == 299792458.0
    assert oracle.eps0() * oracle.mu0() * oracle.c0() ** 2 == pytest.approx(1.0, rel=1e-14)


def test_source_waveform_shape():
    # Modulated Gaussian of section "Modeling Setup": peak envelope at 3 Tp,
    # exp(-1/2) one Tp away, carrier cos(2 pi f0 t).
    f0 = 5e9
    Tp = 1 / f0
    assert oracle.source_value(2.0, f0, Tp, 3 * Tp, 3 * Tp) == pytest.approx(2.0 * math.cos(2 * math.pi * 3), rel=1e-13)
    assert oracle.source_value(1.0, f0, Tp, 3 * Tp, 2 * Tp) == pytest.approx(math.exp(-0.5) * math.cos(4 * math.pi), rel=1e-13)
    t = 1.234e-10
    ref = math.exp(-((t - 3 * Tp) ** 2) / (2 * Tp * Tp)) * math.cos(2 * math.pi * f0 * t)
    assert oracle.source_value(1.0, f0, Tp, 3 * Tp, t) == pytest.approx(ref, rel=1e-13)


# ------------------------------------------------------------ LLG alone
def test_llg_trapezoid_is_exact_rotation_without_damping():
    rng = np.random.default_rng(11)
    for _ in range(20):
        Ms = 1.4e5
        M = rng.normal(size=3)
        M *= Ms / np.linalg.norm(M)
        H = rng.normal(size=3) * 8e4
        kappa = 10 ** rng.uniform(-12, -5)
        out = oracle.llg_trapezoid(M, H, H, kappa, 0.0, Ms)
        ang = cf.cayley_angle(kappa, np.linalg.norm(H))
        ref = cf.rotate(M, H, ang)
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-10 * Ms)
        assert np.linalg.norm(out) == pytest.approx(Ms, rel=1e-14)


def test_llg_damped_matches_continuous_closed_form_second_order():
    # fixed field along +z; theta0 = 60 deg; compare after a fixed time.
    mu0 = cf.MU0
    gamma, H, Ms, alpha = 1.76e11, 8e4, 1.4e5, 0.05
    omega = mu0 * gamma * H
    theta0 = math.pi / 3
    T = 2.0 * 2 * math.pi / omega
    errs = []
    for nsub in (400, 800, 1600):
        h = T / nsub
        kappa = mu0 * gamma * h / 2
        M = Ms * np.array([math.sin(theta0), 0.0, math.cos(theta0)])
        Hv = np.array([0.0, 0.0, H])
        for _ in range(nsub):
            M = oracle.llg_trapezoid(M, Hv, Hv, kappa, alpha, Ms)
        th, ph = cf.damped_precession(theta0, omega, alpha, T)
        ref = Ms * np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        errs.append(np.linalg.norm(M - ref) / Ms)
    assert errs[-1] < 5e-5
    # second order in h
    assert 3.5 < errs[0] / errs[1] < 4.5
    assert 3.5 < errs[1] / errs[2] < 4.5


# -------------------------------------------------- LLG coupled in FDTD
def _magnet_material(Ms=1.4e5, alpha=0.0, gamma=1.76e11):
    return Material(eps_r=1.0, sigma=0.0, Ms=Ms, alpha=alpha, gamma=gamma)


def test_single_cell_precesses_about_bias_plus_half_m0():
    """1x1x1 PEC box: every E edge is in a wall so E = 0, the two faces of each
    axis see -dM/2 each and H_eff = (H0 + M0/2) - M/2.  The trapezoidal step is
    then an exact rotation about G = H0 + M0/2 by 2 atan(kappa |G|) per half step."""
    Ms, gamma = 1.4e5, 1.76e11
    dx = 1e-6
    dt = cf.courant_dt(dx, dx, dx, 0.5)
    h0 = np.array([0.02, -0.03, 0.1]) / cf.MU0
    sim = OracleSim(1, 1, 1, dx, dx, dx, dt, [_magnet_material(Ms)], np.zeros((1, 1, 1)), h0,
                    llg_tol=1e-14, llg_max_iter=50)
    M0 = np.array([0.3, 0.5, 0.8])
    M0 = Ms * M0 / np.linalg.norm(M0)
    sim.set_fields(M=M0.reshape(3, 1, 1, 1))
    nsteps = 500
    sim.run(nsteps)
    G = h0 + 0.5 * M0
    kappa = cf.MU0 * gamma * (dt / 2) / 2
    ref = cf.rotate(M0, G, 2 * nsteps * cf.cayley_angle(kappa, np.linalg.norm(G)))
    np.testing.assert_allclose(sim.M.reshape(3), ref, rtol=0, atol=1e-10 * Ms)
    assert np.abs(sim.Ex).max() == 0 and np.abs(sim.Ey).max() == 0 and np.abs(sim.Ez).max() == 0


def _fit_cos(x):
    """Least-squares cos(w dt) from x[n+1] + x[n-1] = 2 cos(w dt) x[n], applied to
    the first differences so that a constant offset drops out."""
    x = np.diff(np.asarray(x, dtype=np.float64))
    a = x[1:-1]
    b = x[2:] + x[:-2]
    return float(np.dot(a, b) / np.dot(a, a)) / 2.0


def test_two_cell_slab_kittel_frequency():
    """1x1x2 slab of two magnetic cells, bias along x.  E = 0 everywhere; the
    discrete dynamic demagnetising factors are 1/2 on x and y and 3/4 on z for
    the symmetric mode, so the Kittel resonance is
    omega = mu0|gamma| sqrt((H0 + Ms/2)(H0 + 3 Ms/4)); the trapezoidal
    half-steps advance its phase by 2 atan(omega h/2) each."""
    Ms, gamma = 1.4e5, 1.76e11
    dx = 1e-3          # E = 0 here, so dx only sets dt: ~60 steps per period
    dt = cf.courant_dt(dx, dx, dx, 0.5)
    H0 = 0.1 / cf.MU0
    sim = OracleSim(1, 1, 2, dx, dx, dx, dt, [_magnet_material(Ms)], np.zeros((2, 1, 1)), [H0, 0, 0],
                    probes=[(0, 0, 0)], llg_tol=1e-13)
    tilt = 1e-4
    M0 = Ms * np.array([math.sqrt(1 - tilt ** 2), tilt, 0.0])
    sim.set_fields(M=np.repeat(M0.reshape(3, 1, 1, 1), 2, axis=1))
    out = sim.run(3000)
    my = out["probes"][:, 0, 7]
    mz = out["probes"][:, 0, 8]
    omega = cf.kittel_demag_rad_s(gamma, H0, Ms, 0.5, 0.75)
    ref = math.cos(2 * cf.trapezoid_phase(omega, dt / 2))
    assert _fit_cos(my) == pytest.approx(ref, abs=1e-11)
    assert _fit_cos(mz) == pytest.approx(ref, abs=1e-11)
    # the fitted phase per step matches to 1e-7 relative; the trapezoidal phase
    # error (omega h)^2/12 ~ 1e-4 is resolved, so the time discretisation is pinned too
    w_fit = math.acos(_fit_cos(mz)) / dt
    w_ref = 2 * cf.trapezoid_phase(omega, dt / 2) / dt
    assert w_fit == pytest.approx(w_ref, rel=1e-7)
    assert abs(w_fit - omega) / omega > 1e-5


# -------------------------------------------------------------- Maxwell
def test_te101_exact_discrete_dispersion():
    nx, ny, nz = 16, 3, 12
    dx, dy, dz = 1.0e-6, 0.7e-6, 1.3e-6
    dt = cf.courant_dt(dx, dy, dz, 0.7)
    sim = OracleSim(nx, ny, nz, dx, dy, dz, dt, [Material()], np.zeros((nz, ny, nx)), [0, 0, 0],
                    probes=[(5, 1, 4)])
    i = np.arange(nx + 1)
    k = np.arange(nz + 1)
    mode = np.sin(math.pi * k / nz)[:, None, None] * np.sin(math.pi * i / nx)[None, None, :]
    sim.set_fields(Ey=np.broadcast_to(mode, sim.Ey.shape))
    out = sim.run(400)
    ey = np.concatenate([[mode[4, 0, 5]], out["probes"][:, 0, 1]])
    w = cf.yee_cavity_omega((1, 0, 1), (nx * dx, ny * dy, nz * dz), (nx, ny, nz), dt)
    assert _fit_cos(ey) == pytest.approx(math.cos(w * dt), abs=1e-12)
    # and the continuum TE101 frequency within the O((k d)^2) dispersion error
    f_cont = cf.cavity_te_freq_continuum((1, 0, 1), (nx * dx, ny * dy, nz * dz))
    f_disc = w / (2 * math.pi)
    kd2 = (math.pi / nx) ** 2
    assert abs(f_disc - f_cont) / f_cont < kd2 / 12


def test_te_mode_3d_and_dielectric():
    # mode (2,1,1) in a uniform dielectric: Ex + Ez pattern solves the discrete
    # eigenproblem when chosen divergence-free; use the recurrence on the energy
    # of the single mode instead of building it: excite Ez(i,j) = sin sin, TM110.
    nx, ny, nz = 10, 8, 2
    dx, dy, dz = 1e-6, 1.2e-6, 0.8e-6
    eps_r = 4.0
    dt = cf.courant_dt(dx, dy, dz, 0.6)
    sim = OracleSim(nx, ny, nz, dx, dy, dz, dt, [Material(eps_r=eps_r)], np.zeros((nz, ny, nx)), [0, 0, 0],
                    probes=[(3, 2, 1)])
    i = np.arange(nx + 1)
    j = np.arange(ny + 1)
    mode = np.sin(2 * math.pi * j / ny)[:, None] * np.sin(math.pi * i / nx)[None, :]
    sim.set_fields(Ez=np.broadcast_to(mode[None], sim.Ez.shape))
    out = sim.run(300)
    ez = np.concatenate([[mode[2, 3]], out["probes"][:, 0, 2]])
    w = cf.yee_cavity_omega((1, 2, 0), (nx * dx, ny * dy, nz * dz), (nx, ny, nz), dt, eps_r=eps_r)
    assert _fit_cos(ez) == pytest.approx(math.cos(w * dt), abs=1e-12)


def test_first_step_source_injection_sign_and_time():
    """Empty box, zero fields: after one step the source edge holds
    E = -(dt/eps0) J(t = dt/2), the discrete Ampere law with J at half step."""
    n = 6
    dx = 1e-6
    dt = cf.courant_dt(dx, dx, dx, 0.5)
    f0 = 7e9
    src = Source(comp=0, ijk=(2, 3, 3), J0=5.0, f0=f0, Tp=1e-11, tpk=2e-12)
    sim = OracleSim(n, n, n, dx, dx, dx, dt, [Material()], np.zeros((n, n, n)), [0, 0, 0], sources=[src])
    sim.run(1)
    J = oracle.source_value(5.0, f0, 1e-11, 2e-12, 0.5 * dt)
    assert sim.Ex[3, 3, 2] == pytest.approx(-dt / cf.EPS0 * J, rel=1e-13)
    nz_vals = np.count_nonzero(sim.Ex) + np.count_nonzero(sim.Ey) + np.count_nonzero(sim.Ez)
    assert nz_vals == 1


# ------------------------------------------------------------ invariants
def _random_problem(seed, alpha=0.0, sigma=0.0, nx=9, ny=8, nz=7, random_em=True, tilt=0.3, e_scale=50.0):
    rng = np.random.default_rng(seed)
    mats = [Material(eps_r=1.0), Material(eps_r=3.5, sigma=sigma), _magnet_material(1.4e5, alpha),
            _magnet_material(0.9e5, alpha, 1.5e11), Material(pec=True)]
    mid = np.zeros((nz, ny, nx), dtype=np.uint8)
    mid[: nz // 2] = 1
    mid[2:4, 2:5, 3:6] = 2
    mid[4:6, 4:6, 1:3] = 3
    mid[1, 6, 7] = 4
    dx = 1e-6
    dt = cf.courant_dt(dx, 1.1 * dx, 0.9 * dx, 0.5)
    h0 = np.array([0.03, 0.01, 0.08]) / cf.MU0
    sim = OracleSim(nx, ny, nz, dx, 1.1 * dx, 0.9 * dx, dt, mats, mid, h0, llg_tol=1e-12, llg_max_iter=60)
    # random interior E (walls and PEC edges are zeroed by the first E push),
    # random H, M tilted from the bias by up to 0.3 rad
    if random_em:
        sim.set_fields(Ex=rng.normal(size=sim.Ex.shape) * e_scale, Ey=rng.normal(size=sim.Ey.shape) * e_scale,
                       Ez=rng.normal(size=sim.Ez.shape) * e_scale, Hx=rng.normal(size=sim.Hx.shape) * 0.1,
                       Hy=rng.normal(size=sim.Hy.shape) * 0.1, Hz=rng.normal(size=sim.Hz.shape) * 0.1)
    Ms = np.array([m.Ms for m in mats])[mid]
    u = h0 / np.linalg.norm(h0)
    M = np.zeros((3, nz, ny, nx))
    pert = rng.normal(size=(3, nz, ny, nx)) * tilt
    for d in range(3):
        M[d] = u[d] + pert[d]
    M *= Ms / np.linalg.norm(M, axis=0)
    sim.set_fields(M=M)
    # one step to put E in its admissible subspace (walls/PEC at zero)
    sim.run(1)
    return sim


def test_energy_conserved_without_loss():
    """alpha = 0, sigma = 0, no source: field + Zeeman energy is constant up to
    the O((omega dt)^2) oscillation of the leap-frog; no secular drift."""
    sim = _random_problem(3, random_em=False)
    out = sim.run(3000)
    W = out["energy"]
    W0 = W[0]
    assert np.abs(W - W0).max() / abs(W0) < 1e-8
    assert abs(W[-300:].mean() - W[:300].mean()) / abs(W0) < 1e-9


def test_energy_decays_with_damping():
    sim = _random_problem(4, alpha=0.05, random_em=False)
    out = sim.run(1500)
    W = out["energy"]
    assert np.all(np.diff(W) < 0)


def test_energy_decays_with_conductivity():
    sim = _random_problem(4, sigma=2e3, tilt=0.0, e_scale=1e5)
    out = sim.run(600)
    W = out["energy"]
    block = W.reshape(6, 100).mean(axis=1)
    assert np.all(np.diff(block) < 0)
    assert W[-1] < 0.5 * W[0]


def test_div_b_change_stays_at_roundoff():
    sim = _random_problem(5, alpha=0.02)
    d0 = sim.div_b()
    scale = max(np.abs(sim.Hx).max(), np.abs(sim.M).max()) / sim.dx
    sim.run(400)
    d1 = sim.div_b()
    assert np.abs(d1 - d0).max() / scale < 1e-11


def test_magnetisation_norm_held_at_ms():
    sim = _random_problem(6, alpha=0.01)
    sim.run(300)
    Ms = np.array([m.Ms for m in sim.materials])[sim.mat_id]
    nrm = np.linalg.norm(sim.M, axis=0)
    mag = Ms > 0
    np.testing.assert_allclose(nrm[mag], Ms[mag], rtol=1e-13)
    assert np.all(nrm[~mag] == 0)


def test_probe_row_equals_state():
    sim = _random_problem(7)
    sim._probe = np.array([[3, 2, 2], [1, 1, 1]], dtype=np.int32)
    out = sim.run(3)
    p = out["probes"][-1]
    for q, (i, j, k) in enumerate([(3, 2, 2), (1, 1, 1)]):
        vals = [sim.Ex[k, j, i], sim.Ey[k, j, i], sim.Ez[k, j, i], sim.Hx[k, j, i], sim.Hy[k, j, i],
                sim.Hz[k, j, i], sim.M[0, k, j, i], sim.M[1, k, j, i], sim.M[2, k, j, i]]
        np.testing.assert_array_equal(p[q], vals)


def test_llg_iteration_converges_fast_and_fixed_mode_agrees():
    sim = _random_problem(8, alpha=0.01)
    ref = _random_problem(8, alpha=0.01)
    ref.llg_fixed_iter = 6
    out = sim.run(20)
    ref.run(20)
    assert out["iters"].max() <= 4 and out["iters"].min() >= 2
    np.testing.assert_allclose(sim.M, ref.M, rtol=0, atol=1e-9 * 1.4e5)


# ------------------------------------------------------------ brute force
def test_assembled_curls_are_transposes_and_divergence_free():
    geo = YeeGeometry(3, 4, 5, 1.0, 1.3, 0.7)
    CE = geo.curl_on_faces()
    CH = geo.curl_on_edges()
    D = geo.div_on_cells()
    interior = np.array([not geo.is_wall_edge(a, Dd) for a, Dd, e in geo.edges()])
    diff = (CH - CE.T.tocsr()).toarray()[interior]
    scale = np.abs(CE).max()
    assert np.abs(diff).max() <= 1e-15 * scale
    assert np.abs((D @ CE).toarray()).max() <= 1e-15 * scale * np.abs(D).max()
    # structure: every interior edge sees exactly four faces, every face four edges
    assert np.all(np.diff(CH.indptr)[interior] == 4)
    assert np.all(np.diff(CE.indptr) == 4)


def test_oracle_step_equals_assembled_operator_step():
    nx, ny, nz = 3, 4, 5
    dx, dy, dz = 1e-6, 1.3e-6, 0.7e-6
    rng = np.random.default_rng(21)
    eps_cell = rng.uniform(1, 12, size=(nz, ny, nx))
    sig_cell = rng.uniform(0, 5e4, size=(nz, ny, nx))
    pec = np.zeros((nz, ny, nx), dtype=bool)
    pec[3, 1, 2] = True
    # one material per cell so that eps, sigma, PEC differ everywhere
    mats = [Material(eps_r=1.0, sigma=float(sig_cell.ravel()[c]), pec=bool(pec.ravel()[c])) for c in range(nx * ny * nz)]
    mid = np.arange(nx * ny * nz, dtype=np.uint8).reshape(nz, ny, nx)
    dt = cf.courant_dt(dx, dy, dz, 0.5)
    sim = OracleSim(nx, ny, nz, dx, dy, dz, dt, mats, mid, [0, 0, 0], eps_r_cell=eps_cell)
    geo = YeeGeometry(nx, ny, nz, dx, dy, dz)
    step, frozen, _ = maxwell_step_matrices(geo, eps_cell, sig_cell, pec, dt, cf.MU0, cf.EPS0)
    E = rng.normal(size=geo.n_edges)
    E[frozen] = 0.0
    H = rng.normal(size=geo.n_faces) * 1e-3
    Ex, Ey, Ez = geo.unpack_E(E)
    Hx, Hy, Hz = geo.unpack_H(H)
    sim.set_fields(Ex=Ex, Ey=Ey, Ez=Ez, Hx=Hx, Hy=Hy, Hz=Hz)
    for _ in range(3):
        E, H = step(E, H)
    sim.run(3)
    np.testing.assert_allclose(geo.pack_E(sim.Ex, sim.Ey, sim.Ez), E, rtol=1e-12, atol=1e-12 * np.abs(E).max())
    np.testing.assert_allclose(geo.pack_H(sim.Hx, sim.Hy, sim.Hz), H, rtol=1e-12, atol=1e-12 * np.abs(H).max())


def test_magnet_coupling_matches_assembled_mean_operator():
    """With E = 0 and H = 0 at the start of a half-push, the oracle's face field
    after it must equal -A^T (M_new - M_old), A being the assembled
    face-to-cell mean, and the cell field it used must be A H + H0."""
    nx, ny, nz = 4, 3, 3
    dx = 1e-6
    dt = cf.courant_dt(dx, dx, dx, 0.5)
    mats = [Material(), _magnet_material(1.4e5, 0.02)]
    mid = np.zeros((nz, ny, nx), dtype=np.uint8)
    mid[1, 0:2, 1:4] = 1
    mid[2, 1, 2] = 1
    h0 = np.array([0.0, 0.05, 0.08]) / cf.MU0
    sim = OracleSim(nx, ny, nz, dx, dx, dx, dt, mats, mid, h0, llg_tol=1e-14)
    rng = np.random.default_rng(5)
    M = sim.M + rng.normal(size=sim.M.shape) * 2e4 * (mid > 0)
    M *= np.where(mid > 0, 1.4e5 / np.maximum(np.linalg.norm(M, axis=0), 1e-300), 0.0)
    sim.set_fields(M=M)
    Mold = sim.M.copy()
    sim.half_push()
    geo = YeeGeometry(nx, ny, nz, dx, dx, dx)
    A = geo.face_to_cell_mean()
    dM = (sim.M - Mold).reshape(3, -1).ravel()
    H = geo.pack_H(sim.Hx, sim.Hy, sim.Hz)
    np.testing.assert_allclose(H, -(A.T @ dM), rtol=0, atol=1e-12 * np.abs(dM).max())
    # the new M solves the trapezoid with H_eff = A H_new + H0 (converged)
    He1 = (A @ H).reshape(3, -1) + h0[:, None]
    kappa = cf.MU0 * 1.76e11 * (dt / 2) / 2
    for c in np.flatnonzero(mid.ravel() > 0):
        m_new = oracle.llg_trapezoid(Mold.reshape(3, -1)[:, c], h0, He1[:, c], kappa, 0.02, 1.4e5)
        np.testing.assert_allclose(sim.M.reshape(3, -1)[:, c], m_new, rtol=0, atol=1e-9)


def test_coupled_cavity_and_magnet_do_not_gain_energy_at_small_angles():
    """A pulse rings a PEC cavity holding a YIG block (alpha > 0) at tiny
    precession angles, where the change of M per half-push is far below
    tol * Ms.  After the pulse the energy must not grow (Eq. LLG with damping
    and lossless Maxwell: it decays).  Stopping the LLG iteration at the first
    iterate, whose residual against M^n is just the size of the change, keeps
    only the explicit part of the M-H coupling and makes this energy grow
    ~10^4-fold in 3000 steps; the solve must take at least two iterates."""
    from paper_2510_22221_b300 import workloads as W
    from tests.helpers import oracle_from_workload

    w = W.anticrossing_sweep(n_inst=1, b_lo=0.1, b_hi=0.1, steps=3000)[0]
    sim = oracle_from_workload(w)
    out = sim.run(3000)
    E = out["energy"]
    assert out["iters"].min() >= 2
    tail = E[600:].reshape(-1, 200).mean(axis=1)    # the pulse is over by step ~400
    assert np.all(np.diff(tail) <= 1e-12 * tail[0])
    assert E[-1] < E[600]
