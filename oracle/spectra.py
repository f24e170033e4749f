"""FP64 oracle of the spectral post-processing of probe time series (arxiv
2510.22221: the Fourier spectra of E_x behind the anti-crossing maps, section
"Results"; the ESPRIT extraction of the two polariton frequencies and their Q
factors; the hybrid-mode frequencies of Eq. omega_pm).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the product path never
imports it.  Plain numpy, FP64; library routines (matrix product, SVD,
eigenvalues, least squares) serve as steps.  Each function states the
definition it writes out.
"""
from __future__ import annotations

import numpy as np


def window(n: int, kind: str) -> np.ndarray:
    """Rectangular ("rect") or Hann ("hann": 0.5 - 0.5 cos(2 pi t / (n - 1)))."""
    if kind == "rect":
        return np.ones(n)
    if kind == "hann":
        if n == 1:
            return np.ones(1)
        t = np.arange(n)
        return 0.5 - 0.5 * np.cos(2.0 * np.pi * t / (n - 1))
    raise ValueError(kind)


def dft_magnitude(x, dt: float, freqs, kind: str = "hann") -> np.ndarray:
    """|X(f)| = |sum_t w_t x_t exp(-2 pi i f t dt)| at the given frequencies:
    the discrete-time Fourier transform of the windowed series, written as an
    explicit matrix (one row per frequency) times the series."""
    x = np.asarray(x, dtype=np.float64)
    f = np.asarray(freqs, dtype=np.float64)
    t = np.arange(x.size, dtype=np.float64) * dt
    phase = np.exp(-2j * np.pi * np.outer(f, t))
    return np.abs(phase @ (window(x.size, kind) * x))


def block_means(x, d: int):
    """The series of means of consecutive blocks of d samples (the last
    incomplete block dropped): y_b = (x_{bd} + ... + x_{bd+d-1}) / d."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size // d * d
    return x[:n].reshape(-1, d).mean(axis=1)


def matrix_pencil(x, dt: float, order: int, pencil: int | None = None):
    """Complex exponentials z_k^t fitted to a real series by the shift
    invariance of its Hankel data matrix (ESPRIT / matrix pencil):

      Y[m, j] = x[m + j]  (m < n - L, j <= L),  Y = U S V^T (SVD),
      V_s = first `order` right singular vectors,
      Phi = pinv(V_s[:-1]) V_s[1:],  z_k = eigenvalues of Phi,

    then amplitudes c_k from the least-squares Vandermonde fit
    x_t ~ sum_k c_k z_k^t.  Returns (freq, decay, amplitude, Q) of the modes
    with positive frequency, sorted by frequency: f = arg z / (2 pi dt),
    decay rate a = -ln|z| / dt (amplitude ~ exp(-a t)), amplitude 2|c_k| of
    the real cosine, Q = pi f / a."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    L = pencil if pencil else min(n // 3, 200)
    Y = np.lib.stride_tricks.sliding_window_view(x, L + 1)
    _, _, Vt = np.linalg.svd(Y, full_matrices=False)
    Vs = Vt[:order].T
    Phi = np.linalg.pinv(Vs[:-1]) @ Vs[1:]
    z = np.linalg.eigvals(Phi)
    Vand = z[None, :] ** np.arange(n)[:, None]
    c, *_ = np.linalg.lstsq(Vand, x.astype(np.complex128), rcond=None)
    f = np.angle(z) / (2 * np.pi * dt)
    a = -np.log(np.abs(z)) / dt
    keep = f > 0
    f, a, amp = f[keep], a[keep], 2 * np.abs(c[keep])
    idx = np.argsort(f)
    f, a, amp = f[idx], a[idx], amp[idx]
    with np.errstate(divide="ignore"):
        Q = np.where(a != 0, np.pi * f / a, np.inf)
    return f, a, amp, Q


def strongest_in_band(modes, fmin: float, fmax: float, count: int):
    """The `count` modes of largest amplitude with fmin <= f <= fmax, returned
    sorted by frequency (rows of (f, decay, amplitude, Q))."""
    f, a, amp, Q = modes
    sel = np.nonzero((f >= fmin) & (f <= fmax))[0]
    sel = sel[np.argsort(-amp[sel])][:count]
    sel = sel[np.argsort(f[sel])]
    return f[sel], a[sel], amp[sel], Q[sel]


def hybrid_modes(f_p: float, f_m, g: float):
    """Eq. omega_pm (in frequency units): f_pm = f_p + D/2 +- sqrt(D^2 + 4 g^2)/2
    with D = f_m - f_p, so that f_pm = f_p +- g at resonance (splitting 2g)."""
    d = np.asarray(f_m, dtype=np.float64) - f_p
    r = np.sqrt(d * d + 4.0 * g * g) / 2.0
    return f_p + d / 2.0 + r, f_p + d / 2.0 - r


def coupling_fit(f_plus, f_minus):
    """Cavity frequency f_p and coupling g from hybrid-mode pairs measured at
    several detunings, by the relation that Eq. omega_pm implies for
    S = f+ + f- and D = f+ - f-:  D^2 - S^2 = 4 (f_p^2 + g^2) - 4 f_p S,
    linear in the unknowns A = 4 (f_p^2 + g^2), B = -4 f_p; least squares over
    the pairs.  Returns (f_p, g); the splitting at resonance is 2g."""
    fp = np.asarray(f_plus, dtype=np.float64)
    fm = np.asarray(f_minus, dtype=np.float64)
    S, D = fp + fm, fp - fm
    M = np.stack([np.ones_like(S), S], axis=1)
    (A, B), *_ = np.linalg.lstsq(M, D * D - S * S, rcond=None)
    f_c = -B / 4.0
    return f_c, float(np.sqrt(max(A / 4.0 - f_c * f_c, 0.0)))
