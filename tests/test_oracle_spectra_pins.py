"""Pins of the spectral oracle (oracle/spectra.py) against what mathematics
fixes, independently of the oracle's own formulas: library FFT bins,
Parseval's identity, closed-form transforms of a cosine and of a constant,
damped sinusoids with known parameters, and the 2x2 coupled-mode eigenvalue
problem whose eigenvalues Eq. omega_pm writes out."""
import numpy as np
import pytest

from oracle import spectra as S


def test_dft_equals_library_fft_on_the_bin_grid():
    rng = np.random.default_rng(0)
    n, dt = 257, 3e-12
    x = rng.standard_normal(n)
    k = np.arange(n)
    X = S.dft_magnitude(x, dt, k / (n * dt), kind="rect")
    np.testing.assert_allclose(X, np.abs(np.fft.fft(x)), rtol=1e-10, atol=1e-10)


def test_dft_parseval():
    rng = np.random.default_rng(1)
    n, dt = 200, 1e-12
    x = rng.standard_normal(n)
    X = S.dft_magnitude(x, dt, np.arange(n) / (n * dt), kind="rect")
    assert np.sum(X ** 2) == pytest.approx(n * np.sum(x ** 2), rel=1e-12)


def test_dft_of_a_cosine_on_a_bin_and_of_a_constant():
    n, dt, k0 = 400, 2e-12, 37
    t = np.arange(n)
    x = np.cos(2 * np.pi * k0 * t / n)
    X = S.dft_magnitude(x, dt, np.array([k0, k0 + 3, 5]) / (n * dt), kind="rect")
    np.testing.assert_allclose(X, [n / 2, 0.0, 0.0], atol=1e-9 * n)
    # sum of the symmetric Hann window: n/2 - (1/2) sum_t cos(2 pi t/(n-1)) = (n-1)/2
    assert S.dft_magnitude(np.ones(n), dt, [0.0], kind="hann")[0] == pytest.approx((n - 1) / 2, rel=1e-12)


def test_matrix_pencil_recovers_damped_cosines():
    dt = 5e-12
    n = 3000
    t = np.arange(n) * dt
    f = np.array([2.61e9, 2.93e9, 7.4e9])
    a = np.array([3.0e6, 1.2e7, 5.0e7])
    A = np.array([1.0, 0.6, 0.25])
    ph = np.array([0.3, -1.1, 2.0])
    x = sum(A[q] * np.exp(-a[q] * t) * np.cos(2 * np.pi * f[q] * t + ph[q]) for q in range(3))
    fr, de, amp, Q = S.matrix_pencil(x, dt, order=6)
    np.testing.assert_allclose(fr, f, rtol=1e-9)
    np.testing.assert_allclose(de, a, rtol=1e-5)
    np.testing.assert_allclose(amp, A, rtol=1e-7)
    np.testing.assert_allclose(Q, np.pi * f / a, rtol=1e-5)
    # selection: the two strongest modes in a band, by frequency
    sf, _, samp, _ = S.strongest_in_band((fr, de, amp, Q), 2e9, 8e9, 2)
    np.testing.assert_allclose(sf, f[:2], rtol=1e-9)
    np.testing.assert_allclose(samp, A[:2], rtol=1e-7)


def test_block_means_keep_frequency_and_decay():
    """Block means of d samples of A z^t are A (1 - z^d) / (d (1 - z)) (z^d)^b:
    the same frequency and decay at step d dt, with that amplitude factor
    (a geometric sum), which the pencil fit then recovers."""
    dt, d, n = 1e-12, 20, 20000
    f, a, A = 2.7e9, 3e6, 1.3
    t = np.arange(n) * dt
    x = A * np.exp(-a * t) * np.cos(2 * np.pi * f * t)
    y = S.block_means(x, d)
    assert y.shape == (n // d,)
    z = np.exp((-a + 2j * np.pi * f) * dt)
    fac = (1 - z ** d) / (d * (1 - z))
    b = np.arange(n // d)
    np.testing.assert_allclose(y, A * np.real(fac * z ** (d * b)), rtol=0, atol=1e-12 * A)
    fr, de, amp, q = S.matrix_pencil(y, d * dt, 2, 200)
    assert fr[0] == pytest.approx(f, rel=1e-10)
    assert de[0] == pytest.approx(a, rel=1e-6)
    assert amp[0] == pytest.approx(A * abs(fac), rel=1e-8)


def test_hybrid_modes_are_the_coupled_mode_eigenvalues():
    f_p, g = 15.2e9, 0.335e9
    f_m = np.linspace(13.5e9, 17.0e9, 11)
    fp_, fm_ = S.hybrid_modes(f_p, f_m, g)
    for q, m in enumerate(f_m):
        lo, hi = np.linalg.eigvalsh(np.array([[f_p, g], [g, m]]))
        assert fp_[q] == pytest.approx(hi, rel=1e-14)
        assert fm_[q] == pytest.approx(lo, rel=1e-14)
    # on resonance the pair is f_p -+ g: splitting 2g
    hi, lo = S.hybrid_modes(f_p, f_p, g)
    assert hi - lo == pytest.approx(2 * g, rel=1e-14)


def test_coupling_fit_recovers_cavity_frequency_and_g():
    f_p, g = 2.83e9, 0.21e9
    f_m = np.linspace(1.4e9, 4.2e9, 9)
    fp_, fm_ = S.hybrid_modes(f_p, f_m, g)
    fc, gf = S.coupling_fit(fp_, fm_)
    assert fc == pytest.approx(f_p, rel=1e-12)
    assert gf == pytest.approx(g, rel=1e-10)
