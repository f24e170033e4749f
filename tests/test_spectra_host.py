"""Host-side mode fits of the library (ESPRIT, coupling fit) against the FP64
spectral oracle on the same series.  These entry points run on the host in
FP64 and need no GPU.  The two sides take different routes to the same
definition: the library builds the Hankel Gram matrix by its shift recursion
and diagonalises it by Jacobi rotations, then finds the eigenvalues of the
shift operator by Hessenberg QR; the oracle takes the SVD of the Hankel
matrix itself and library eigenvalues."""
import numpy as np
import pytest

import paper_2510_22221_b300 as pkg
from oracle import spectra as S


def damped(dt, n, f, a, A, ph):
    t = np.arange(n) * dt
    return sum(A[q] * np.exp(-a[q] * t) * np.cos(2 * np.pi * f[q] * t + ph[q]) for q in range(len(f)))


@pytest.mark.parametrize("pencil", [0, 64, 200, 400])
def test_fit_modes_matches_oracle_clean(pencil):
    dt, n = 4e-12, 2400
    f, a = np.array([2.61e9, 2.93e9, 7.4e9]), np.array([3e6, 1.2e7, 5e7])
    A, ph = np.array([1.0, 0.6, 0.25]), np.array([0.3, -1.1, 2.0])
    x = damped(dt, n, f, a, A, ph)
    fr, de, amp, q = pkg.fit_modes(x, dt, 6, pencil=pencil)
    of, oa, oamp, oq = S.matrix_pencil(x, dt, 6, pencil or None)
    np.testing.assert_allclose(fr, of, rtol=1e-11)
    np.testing.assert_allclose(de, oa, rtol=1e-7)
    np.testing.assert_allclose(amp, oamp, rtol=1e-9)
    np.testing.assert_allclose(q, oq, rtol=1e-7)
    np.testing.assert_allclose(fr, f, rtol=1e-9)   # and both recover the truth


@pytest.mark.parametrize("seed", [0, 1])
def test_fit_modes_matches_oracle_noisy_band_selection(seed):
    rng = np.random.default_rng(seed)
    dt, n = 5e-12, 3000
    f, a = np.array([2.55e9, 2.98e9, 3.3e9, 9.1e9]), np.array([2e6, 4e6, 9e7, 1e7])
    A, ph = np.array([0.8, 1.0, 0.05, 2.0]), rng.uniform(-3, 3, 4)
    x = damped(dt, n, f, a, A, ph) + 1e-3 * rng.standard_normal(n)
    got = pkg.fit_modes(x, dt, 16, pencil=300, fmin=2e9, fmax=3.5e9, max_modes=2)
    ref = S.strongest_in_band(S.matrix_pencil(x, dt, 16, 300), 2e9, 3.5e9, 2)
    np.testing.assert_allclose(got[0], ref[0], rtol=1e-9)
    np.testing.assert_allclose(got[2], ref[2], rtol=1e-6)
    np.testing.assert_allclose(got[0], f[:2], rtol=1e-5)


def test_fit_modes_with_block_means_matches_oracle():
    """The library's decimated fit is the oracle's pencil fit of the block
    means (same series, same settings)."""
    rng = np.random.default_rng(4)
    dt, n, d = 7.6e-13, 8000, 20
    f, a = np.array([2.41e9, 2.77e9, 3.9e9, 40e9]), np.array([2e6, 4e6, 3e7, 1e8])
    A, ph = np.array([0.3, 1.0, 0.2, 0.5]), rng.uniform(-3, 3, 4)
    x = damped(dt, n, f, a, A, ph) + 1e-4 * rng.standard_normal(n)
    got = pkg.fit_modes(x, dt, 24, pencil=100, fmin=1.5e9, fmax=4.5e9, max_modes=2, decimate=d)
    ref = S.strongest_in_band(S.matrix_pencil(S.block_means(x, d), d * dt, 24, 100), 1.5e9, 4.5e9, 2)
    np.testing.assert_allclose(got[0], ref[0], rtol=1e-9)
    np.testing.assert_allclose(got[0], f[:2], rtol=1e-5)


def test_fit_coupling_matches_oracle():
    f_m = np.linspace(1.9e9, 3.7e9, 7)
    fp_, fm_ = S.hybrid_modes(2.79e9, f_m, 0.23e9)
    rng = np.random.default_rng(4)
    fp_ = fp_ * (1 + 1e-6 * rng.standard_normal(7))
    fm_ = fm_ * (1 + 1e-6 * rng.standard_normal(7))
    got = pkg.fit_coupling(fp_, fm_)
    ref = S.coupling_fit(fp_, fm_)
    assert got[0] == pytest.approx(ref[0], rel=1e-12)
    assert got[1] == pytest.approx(ref[1], rel=1e-9)


def test_fit_argument_errors():
    x = np.ones(100)
    with pytest.raises(pkg.LLGError):
        pkg.fit_modes(x, 0.0, 4)
    with pytest.raises(pkg.LLGError):
        pkg.fit_modes(x, 1e-12, 4, pencil=99)
    with pytest.raises(pkg.LLGError):
        pkg.fit_coupling([1.0], [0.5])
    with pytest.raises(pkg.LLGError):
        pkg.fit_coupling([2.0, 2.0], [1.0, 1.0])
