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
absorbed power from Eq. S1.  layered_field solves the same equations for
the cavity a PEC-walled solver can hold: walls of either kind and fields of
Eq. S7 times a fixed transverse sine (a guided mode, k^2 -> k^2 - kt^2);
cavity_poles gives the resonances of the absorbed power as the complex
poles of chi with that solve's coupling.

Readings (the supplement leaves them open):
  * the film is centred in the cavity (the phases of the printed Eq. S10
    coefficients, arg = -k d3 / 2, point there);
  * eps_r of the film is 1: the printed k^m = 297.033 + 0.188 i m^-1 at
    14.17 GHz follows with eps_r = 1 and sigma = 1e-3 S/m, not with the
    tabulated 7.1 (which gives 791 m^-1);
  * w_m is the Kittel frequency gamma' sqrt(H (H + Ms)) of the tabulated
    gamma' and Ms at 1800 Oe (14.1726 GHz, printed 14.17).
The printed k^m and the Kittel frequency are reproduced, and the printed
<theta_zy> = 4.966e9 Hz is the film mean of Eq. S8's form evaluated on the
printed Eq. S10 coefficients (real part to 7e-4).  Those coefficients are,
though, a common 2.29 % above this solve's (same phases), and that excess
is the whole printed coupling: the solve itself gives ~1.36e7 Hz, so the
printed value stays unreproduced from the stated inputs (parity of the
solve's <theta_zy> against the printed number unpinned).
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
    return layered_field(w, d1, d2, d3, eps_m, eps_c, sigma_m, sigma_c, M)[:5]


def layered_field(w: float, d1: float, d2: float, L: float, eps_m: float, eps_c: float, sigma_m: float,
                  sigma_c: float, M: float = 1.0, kt: float = 0.0, walls: str = "pmc"):
    """Eqs. S7-S9 for a film [d1, d2] in a cavity [0, L], in the two forms a
    closed cavity allows.  The fields are those of Eq. S7 times a fixed
    transverse profile of wavenumber kt (a guided mode: for kt = 0 the
    supplement's plane fields), so that in each layer
        H'' + kappa^2 H = -kappa^2 M,   kappa^2 = k^2 - kt^2,
    and the tangential E continuous at an interface is (iw mu0 / kappa^2) H'
    (at kt = 0 the supplement's (sigma - i eps w)^-1 H').  walls = "pmc": H =
    0 at 0 and L, the supplement's cavity; walls = "pec": tangential E = 0,
    so H' = 0, and the cavity field is A cos(kappa z) below the film and
    B cos(kappa (L - z)) above it.  Returns (A, B, C, D, mean film H,
    determinant of the 4 x 4 system); the determinant vanishes at the
    cavity's resonances with M = 0."""
    if walls not in ("pmc", "pec"):
        raise ValueError("walls: 'pmc' or 'pec'")
    km = np.sqrt(wavenumber(w, eps_m, sigma_m) ** 2 - kt * kt)
    kc = np.sqrt(wavenumber(w, eps_c, sigma_c) ** 2 - kt * kt)
    # the interface weight kappa^2 / (i w mu0): H' / weight is continuous
    ym, yc = km * km / (1j * w * MU0), kc * kc / (1j * w * MU0)
    e = np.exp
    if walls == "pmc":
        lo, dlo = np.sin(kc * d1), kc * np.cos(kc * d1)                    # A sin(kc z) and its slope at d1
        hi, dhi = np.sin(kc * (L - d2)), -kc * np.cos(kc * (L - d2))      # B sin(kc (L - z)) at d2
    else:
        lo, dlo = np.cos(kc * d1), -kc * np.sin(kc * d1)
        hi, dhi = np.cos(kc * (L - d2)), kc * np.sin(kc * (L - d2))
    A = np.array([
        [lo, 0, -e(1j * km * d1), -e(-1j * km * d1)],
        [0, hi, -e(1j * km * d2), -e(-1j * km * d2)],
        [dlo / yc, 0, -1j * km * e(1j * km * d1) / ym, 1j * km * e(-1j * km * d1) / ym],
        [0, dhi / yc, -1j * km * e(1j * km * d2) / ym, 1j * km * e(-1j * km * d2) / ym],
    ], dtype=complex)
    rhs = np.array([-M, -M, 0, 0], dtype=complex)
    a, b, c, d = np.linalg.solve(A, rhs)
    return a, b, c, d, film_mean(c, d, km, d1, d2, M), np.linalg.det(A)


def film_mean(c: complex, d: complex, km: complex, d1: float, d2: float, M: float) -> complex:
    """The film's mean field of Eq. S8's form C e^{i k z} + D e^{-i k z} - M
    over [d1, d2] (the average that Eq. S13 takes, times gamma, as the
    coupling)."""
    e = np.exp
    return (c * (e(1j * km * d2) - e(1j * km * d1)) - d * (e(-1j * km * d2) - e(-1j * km * d1))) / (1j * km) / (d2 - d1) - M


def theta_zy(w: float, H: float, p=TABLE_S1, eps_m: float = 1.0, d1: float | None = None) -> complex:
    """<theta_zy> of Eq. S13: gamma times the film's mean H_y per unit m_y
    (M_y = Ms m_y), the film centred unless d1 is given."""
    t, d3 = p["thickness"], p["d3"]
    d1 = (d3 - t) / 2 if d1 is None else d1
    *_, mean = film_field(w, d1, d1 + t, d3, eps_m, p["eps_c"], p["sigma_m"], p["sigma_c"], M=p["Ms"])
    return p["gamma"] * mean


def chi(w: float, H: float, theta: complex, p=TABLE_S1, demag: float = 1.0) -> np.ndarray:
    """Eq. S5b: gamma [[i w, 0, 0], [0, i w, A23], [0, A32 - theta_zy, i w]]^-1
    [[0, 0, 0], [0, 0, -1], [0, 1, 0]] with A23 = i alpha w - gamma H -
    gamma Ms and A32 = -i alpha w + gamma H (Eq. S4a; theta_zx = theta_zz = 0).
    demag scales the film-normal Ms term of A23 (1 for the supplement's
    continuous film)."""
    g, al, Ms = p["gamma"], p["alpha"], p["Ms"]
    a23 = 1j * al * w - g * H - g * demag * Ms
    a32 = -1j * al * w + g * H
    L = np.array([[1j * w, 0, 0], [0, 1j * w, a23], [0, a32 - theta, 1j * w]], dtype=complex)
    R = np.array([[0, 0, 0], [0, 0, -1], [0, 1, 0]], dtype=complex)
    return g * np.linalg.solve(L, R)


def p_abs(w: float, H: float, theta: complex, p=TABLE_S1, demag: float = 1.0) -> float:
    """Eq. S1 up to a constant: Im(h^T chi h) for the tabulated drive h."""
    h = np.asarray(p["h0"], dtype=complex)
    return float(np.imag(h @ chi(w, H, theta, p, demag) @ h))


def s3_determinant(w: complex, H: float, theta: complex, p=TABLE_S1, demag: float = 1.0) -> complex:
    """The determinant of the y-z block of the S3 matrix of Eq. S5b, signed
    so that it reads w^2 - (gamma (H + demag Ms) - i alpha w) (gamma H -
    i alpha w - theta): its zeros in complex w are the poles of chi, the
    resonances of the absorbed power (peak Re w, half-width -Im w)."""
    g, al, Ms = p["gamma"], p["alpha"], p["Ms"]
    a23 = 1j * al * w - g * H - g * demag * Ms
    a32 = -1j * al * w + g * H
    return -((1j * w) * (1j * w) - a23 * (a32 - theta))


def _secant(f, z0: complex, z1: complex, tol: float, maxit: int) -> complex:
    f0, f1 = f(z0), f(z1)
    for _ in range(maxit):
        z2 = z1 - f1 * (z1 - z0) / (f1 - f0)
        if abs(z2 - z1) <= tol * abs(z2):
            return z2
        z0, f0, z1, f1 = z1, f1, z2, f(z2)
    raise RuntimeError("secant iteration did not converge")


def cavity_poles(H: float, d1: float, d2: float, L: float, guesses, p=TABLE_S1, eps_m: float = 1.0,
                 kt: float = 0.0, walls: str = "pmc", demag: float = 1.0, tol: float = 1e-14):
    """The poles of chi with the film's own cavity field as the coupling:
    theta_zy(w) = gamma <H_y>(w) per unit m_y from layered_field (M = Ms),
    inserted in Eq. S5b.  theta has poles at the bare cavity resonances, so
    the zeros are sought of s3_determinant times the 4 x 4 determinant
    (analytic in w), by secant steps from each guess (angular frequencies),
    each later zero with the earlier ones divided out.  Time factor
    exp(-i w t): a resonance decays as exp(Im w t).  Returned sorted by
    Re w."""
    def g(w):
        *_, mean, det = layered_field(w, d1, d2, L, eps_m, p["eps_c"], p["sigma_m"], p["sigma_c"], M=p["Ms"],
                                      kt=kt, walls=walls)
        return s3_determinant(w, H, p["gamma"] * mean, p, demag) * det

    roots = []
    for w0 in guesses:
        def f(w, r=tuple(roots)):
            return g(w) / np.prod([w - x for x in r]) if r else g(w)
        roots.append(_secant(f, complex(w0), complex(w0) * (1 + 1e-6), tol, 200))
    return np.array(sorted(roots, key=lambda z: z.real))
