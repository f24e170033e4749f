"""Pins of the oracle's 1-D analytic magnon-photon cavity (Supplementary
Information, Eqs. S1-S13, Table S1; oracle/supplement.py)."""
import numpy as np
import pytest

from oracle import supplement as S

P = S.TABLE_S1
W_M = S.kittel_w(1800 * S.OE, P["Ms"], P["gamma"])


def test_kittel_frequency_of_the_supplement():
    """14.17 GHz at 1800 Oe with gamma' = 2.23e5 and Ms = 9.7e5 A/m (printed
    after Eq. S10)."""
    assert W_M / (2 * np.pi) == pytest.approx(14.17e9, abs=0.005e9)


def test_film_wavenumber_as_printed():
    """k^m = 297.033 + 0.188 i m^-1 at w_m (printed with Eq. S10), from
    k^2 = eps0 eps_r mu0 w^2 + i sigma mu0 w with sigma = 1e-3 S/m and
    eps_r = 1 (the tabulated eps_r^m = 7.1 would give 791.5 m^-1).  To 2e-5
    relative: w_m rests on the printed Ms, gamma' and the oersted, whose
    rounding moves it by about that much (computed 297.0365)."""
    k = S.wavenumber(W_M, 1.0, P["sigma_m"])
    assert k.real == pytest.approx(297.033, rel=2e-5)
    assert k.imag == pytest.approx(0.188, abs=5e-4)
    assert S.wavenumber(W_M, P["eps_m"], P["sigma_m"]).real == pytest.approx(791.5, abs=0.1)


@pytest.mark.parametrize("z0", [0.5e-3, 1.835e-3, 3.0e-3])
def test_thin_film_field_equals_the_cavity_greens_function(z0):
    """For a film thin against the wavelength, Eq. S7 with the PMC walls is
    the cavity Green's function G(z, z') = sin(k z<) sin(k (d3 - z>)) /
    (k sin(k d3)) driven by k^2 M over the film: <H> = k M t sin(k z0)
    sin(k (d3 - z0)) / sin(k d3) to first order in k t; the boundary-value
    solve of Eqs. S8-S9 (a 4 x 4 system) agrees to 1e-3."""
    t, d3 = P["thickness"], P["d3"]
    k = S.wavenumber(W_M, 1.0, P["sigma_m"])
    *_, mean = S.film_field(W_M, z0 - t / 2, z0 + t / 2, d3, 1.0, 1.0, P["sigma_m"], P["sigma_c"], M=1.0)
    closed = k * t * np.sin(k * z0) * np.sin(k * (d3 - z0)) / np.sin(k * d3)
    assert abs(mean - closed) < 1e-3 * abs(closed)


def test_printed_wave_coefficients_place_the_film_at_the_centre():
    """The printed Eq. S10 coefficients (424551 - 257055 i) and
    (424224 + 256900 i) per unit m_y have phases -0.5446 and +0.5446 rad:
    -/+ k d3 / 2, the film centred; the solve gives the same phases (their
    magnitudes print 2.3 % above Ms / 2, which the model does not explain)."""
    t, d3 = P["thickness"], P["d3"]
    _, _, c, d, _ = S.film_field(W_M, (d3 - t) / 2, (d3 + t) / 2, d3, 1.0, 1.0, P["sigma_m"], P["sigma_c"],
                                 M=P["Ms"])
    assert np.angle(c) == pytest.approx(np.angle(424551 - 257055j), abs=2e-3)
    assert np.angle(d) == pytest.approx(np.angle(424224 + 256900j), abs=2e-3)


def test_uncoupled_susceptibility_peaks_at_the_kittel_frequency():
    """With theta_zy = 0 the absorbed power of Eq. S1 for the drive h_y peaks
    at the Kittel frequency, with the Gilbert linewidth ~ alpha (2H + Ms)
    gamma."""
    H = 1800 * S.OE
    w = np.linspace(0.95, 1.05, 4001) * W_M
    pa = np.array([S.p_abs(x, H, 0.0) for x in w])
    assert w[np.argmax(pa)] == pytest.approx(W_M, rel=2e-4)
    half = w[pa >= pa.max() / 2]
    fwhm = half[-1] - half[0]
    assert fwhm == pytest.approx(P["alpha"] * (2 * H + P["Ms"]) * P["gamma"], rel=0.05)


def test_coupling_shifts_the_resonance_as_the_linearised_llg_says():
    """A coupling theta_zy enters Eq. S5b as A32 - theta: the resonance moves
    to gamma sqrt((H + Ms) (H - theta / gamma)) (the determinant of the S3
    matrix at alpha = 0)."""
    H = 1800 * S.OE
    p0 = dict(P, alpha=1e-5)
    theta = 0.02 * P["gamma"] * H
    w_c = P["gamma"] * np.sqrt((H + P["Ms"]) * (H - theta / P["gamma"]))
    w = np.linspace(0.97, 1.01, 8001) * W_M
    pa = np.array([abs(S.p_abs(x, H, theta, p0)) for x in w])
    assert w[np.argmax(pa)] == pytest.approx(w_c, rel=2e-5)
