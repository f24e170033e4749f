"""FP64 oracle of the paper's 1-D analytic model of a hybrid magnon-photon
cavity (Supplementary Information, Eqs. S1-S13, Table S1).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.  Plain numpy, FP64;
a 4 x 4 linear solve and a 3 x 3 inverse serve as steps.

The model: fields vary only along z; a film of thickness d2 - d1 magnetised
along x by the bias sits in a cavity 0 < z < d3 closed by perfect magnetic
conductors (tangential H = 0).  Eq. S7 gives, with time factor exp(-i w t),
    H_i'' + k^2 H_i = -k^2 M_i,   k^2 = eps0 eps_r mu0 w^2 + i sigma mu0 w,
solved by Eqs. S8 (forward and backward waves, minus M in the film), with
E_i ~ (sigma - i eps0 eps_r w)^-1 (-dH_j/dz) from Eq. S9 continuous with H at
z = d1, d2.  The film's mean field per unit m_y, times gamma, is the coupling
<theta_zy> (Eq. S13); the susceptibility follows from Eq. S5b and the
absorbed power from Eq. S1.

Readings (the supplement leaves them open):
  * the film is centred in the cavity (the phases of the printed Eq. S10
    coefficients, arg = -k d3 / 2, point there);
  * eps_r of the film is 1: the printed k^m = 297.033 + 0.188 i m^-1 at
    14.17 GHz follows with eps_r = 1 and sigma = 1e-3 S/m, not with the
    tabulated 7.1 (which gives 791 m^-1);
  * w_m is the Kittel frequency gamma' sqrt(H (H + Ms)) of the tabulated
    gamma' and Ms at 1800 Oe (14.1726 GHz, printed 14.17).
Parity of <theta_zy> is unpinned: for the stated sizes the solve (and its
thin-film closed form) gives ~1.36e7 Hz, far from the printed 4.966e9 Hz;
the printed k^m and the Kittel frequency are reproduced.
"""
from __future__ import annotations

import numpy as np

MU0 = 4e-7 * np.pi
C0 = 299792458.0
EPS0 = 1.0 / (MU0 * C0 * C0)
OE = 1e3 / (4 * np.pi)          # one oersted in A/m

# Table S1
TABLE_S1 = dict(sigma_m=1e-3, sigma_c=1e-3, eps_m=7.1, eps_c=1.0, Ms=9.7e5, gamma=2.23e5, alpha=0.003,
                thickness=7e-7, d3=3.67e-3, h0=(0.0, 1e3, 0.0))


def wavenumber(w: float, eps_r: float, sigma: float) -> complex:
    """k of Eq. S7: k^2 = eps0 eps_r mu0 w^2 + i sigma mu0 w (Im k >= 0)."""
    k = np.sqrt(complex(EPS0 * eps_r * MU0 * w * w, sigma * MU0 * w))
    return k if k.imag >= 0 else -k


def kittel_w(H: float, Ms: float, gamma: float) -> float:
    """Angular Kittel frequency of an in-plane film, gamma sqrt(H (H + Ms))
    (the zero of det of the S3 matrix without coupling)."""
    return gamma * np.sqrt(H * (H + Ms))


def film_field(w: float, d1: float, d2: float, d3: float, eps_m: float, eps_c: float, sigma_m: float,
               sigma_c: float, M: float = 1.0):
    """The boundary-value solve of Eqs. S8-S9 for one in-plane component with
    film magnetisation M (uniform): cavity H = A sin(k_c z) below the film
    and B sin(k_c (d3 - z)) above it (PMC walls), film H = C e^{i k_m z} +
    D e^{-i k_m z} - M; H and (sigma - i eps w)^-1 dH/dz continuous at d1 and
    d2.  Returns (A, B, C, D, mean film H)."""
    km, kc = wavenumber(w, eps_m, sigma_m), wavenumber(w, eps_c, sigma_c)
    ym, yc = sigma_m - 1j * EPS0 * eps_m * w, sigma_c - 1j * EPS0 * eps_c * w
    e = np.exp
    A = np.array([
        [np.sin(kc * d1), 0, -e(1j * km * d1), -e(-1j * km * d1)],
        [0, np.sin(kc * (d3 - d2)), -e(1j * km * d2), -e(-1j * km * d2)],
        [kc * np.cos(kc * d1) / yc, 0, -1j * km * e(1j * km * d1) / ym, 1j * km * e(-1j * km * d1) / ym],
        [0, -kc * np.cos(kc * (d3 - d2)) / yc, -1j * km * e(1j * km * d2) / ym, 1j * km * e(-1j * km * d2) / ym],
    ], dtype=complex)
    rhs = np.array([-M, -M, 0, 0], dtype=complex)
    a, b, c, d = np.linalg.solve(A, rhs)
    mean = (c * (e(1j * km * d2) - e(1j * km * d1)) - d * (e(-1j * km * d2) - e(-1j * km * d1))) / (1j * km) / (d2 - d1) - M
    return a, b, c, d, mean


def theta_zy(w: float, H: float, p=TABLE_S1, eps_m: float = 1.0, d1: float | None = None) -> complex:
    """<theta_zy> of Eq. S13: gamma times the film's mean H_y per unit m_y
    (M_y = Ms m_y), the film centred unless d1 is given."""
    t, d3 = p["thickness"], p["d3"]
    d1 = (d3 - t) / 2 if d1 is None else d1
    *_, mean = film_field(w, d1, d1 + t, d3, eps_m, p["eps_c"], p["sigma_m"], p["sigma_c"], M=p["Ms"])
    return p["gamma"] * mean


def chi(w: float, H: float, theta: complex, p=TABLE_S1) -> np.ndarray:
    """Eq. S5b: gamma [[i w, 0, 0], [0, i w, A23], [0, A32 - theta_zy, i w]]^-1
    [[0, 0, 0], [0, 0, -1], [0, 1, 0]] with A23 = i alpha w - gamma H -
    gamma Ms and A32 = -i alpha w + gamma H (Eq. S4a; theta_zx = theta_zz = 0)."""
    g, al, Ms = p["gamma"], p["alpha"], p["Ms"]
    a23 = 1j * al * w - g * H - g * Ms
    a32 = -1j * al * w + g * H
    L = np.array([[1j * w, 0, 0], [0, 1j * w, a23], [0, a32 - theta, 1j * w]], dtype=complex)
    R = np.array([[0, 0, 0], [0, 0, -1], [0, 1, 0]], dtype=complex)
    return g * np.linalg.solve(L, R)


def p_abs(w: float, H: float, theta: complex, p=TABLE_S1) -> float:
    """Eq. S1 up to a constant: Im(h^T chi h) for the tabulated drive h."""
    h = np.asarray(p["h0"], dtype=complex)
    return float(np.imag(h @ chi(w, H, theta, p) @ h))
