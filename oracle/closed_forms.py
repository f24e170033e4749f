"""Closed-form results that pin the FP64 oracle (test infrastructure only).

Each function states a textbook or paper result in its own terms; none of
them calls the oracle's stepping code.
"""
from __future__ import annotations

import math

import numpy as np

MU0 = 4e-7 * math.pi            # vacuum permeability used throughout (H/m)
C0 = 299792458.0                # speed of light (m/s)
EPS0 = 1.0 / (MU0 * C0 * C0)    # vacuum permittivity (F/m)
OE_TO_A_PER_M = 1000.0 / (4.0 * math.pi)


def courant_dt(dx: float, dy: float, dz: float, cfl: float) -> float:
    """3-D Courant step scaled by the CFL factor (section "Modeling Setup":
    CFL 0.9 on a 5 x 19 x 1 um mesh gives 2.94e-15 s)."""
    return cfl / (C0 * math.sqrt(dx ** -2 + dy ** -2 + dz ** -2))


def kittel_cgs_hz(H0_oe: float, four_pi_Ms_gauss: float, gamma_over_2pi_hz_per_oe: float = 2.8e6) -> float:
    """In-plane thin-film Kittel frequency f = (gamma/2pi) sqrt(H0 (H0 + 4 pi Ms))
    in Gaussian units (section "Numerically Predicted ... Coupling": 15.027 GHz
    at 2050 Oe with 4 pi Ms = 1.2e4 G)."""
    return gamma_over_2pi_hz_per_oe * math.sqrt(H0_oe * (H0_oe + four_pi_Ms_gauss))


def kittel_si_hz(H0_a_per_m: float, Ms: float, gamma_prime: float) -> float:
    """omega_m = gamma' sqrt(H0 (H0 + Ms)), gamma' in Hz m/A (rad/s per A/m) as in
    Table S1 (supplement: 14.17 GHz at 1800 Oe, Ms = 9.7e5 A/m, gamma' = 2.23e5)."""
    return gamma_prime * math.sqrt(H0_a_per_m * (H0_a_per_m + Ms)) / (2.0 * math.pi)


def kittel_demag_rad_s(gamma_abs: float, H0: float, Ms: float, n1: float, n2: float) -> float:
    """Kittel resonance of a uniformly magnetised body with dynamic demagnetising
    factors n1, n2 on the two axes transverse to the bias (SI, H in A/m):
    omega = mu0 |gamma| sqrt((H0 + n1 Ms)(H0 + n2 Ms))."""
    return MU0 * gamma_abs * math.sqrt((H0 + n1 * Ms) * (H0 + n2 * Ms))


def trapezoid_phase(omega: float, h: float) -> float:
    """Phase advanced by one trapezoidal (Cayley) substep of length h on a linear
    oscillator of angular frequency omega: 2 atan(omega h / 2)."""
    return 2.0 * math.atan(0.5 * omega * h)


def cayley_angle(kappa: float, H: float) -> float:
    """Rotation angle of the implicit-midpoint precession step M' - M = -kappa (M'+M) x H:
    a rotation about H by 2 atan(kappa |H|)."""
    return 2.0 * math.atan(kappa * H)


def rotate(v: np.ndarray, axis: np.ndarray, angle: float) -> np.ndarray:
    """Rodrigues rotation of v about unit axis by angle (right-handed)."""
    a = axis / np.linalg.norm(axis)
    return v * math.cos(angle) + np.cross(a, v) * math.sin(angle) + a * np.dot(a, v) * (1 - math.cos(angle))


def damped_precession(theta0: float, omega: float, alpha: float, t: float):
    """Continuous LLG dM/dt = -mu0|gamma| M x H + (alpha/Ms) M x dM/dt for a fixed
    field along +z, omega = mu0 |gamma| H.  Polar angle and azimuth:
    phi = omega t / (1 + alpha^2),
    tan(theta/2) = tan(theta0/2) exp(-alpha omega t / (1 + alpha^2))."""
    phi = omega * t / (1.0 + alpha * alpha)
    theta = 2.0 * math.atan(math.tan(0.5 * theta0) * math.exp(-alpha * omega * t / (1.0 + alpha * alpha)))
    return theta, phi


def yee_cavity_omega(mode, lengths, cells, dt: float, eps_r: float = 1.0) -> float:
    """Exact discrete dispersion of the Yee leap-frog scheme for the PEC-box
    eigenmode with mode numbers (m, n, p): with k_i = m_i pi / L_i,
    sin^2(omega dt / 2) / (v dt)^2 = sum_i sin^2(k_i d_i / 2) / d_i^2,
    v = c / sqrt(eps_r)."""
    v = C0 / math.sqrt(eps_r)
    s = 0.0
    for m, L, n in zip(mode, lengths, cells):
        d = L / n
        k = m * math.pi / L
        s += math.sin(0.5 * k * d) ** 2 / d ** 2
    return 2.0 / dt * math.asin(v * dt * math.sqrt(s))


def cavity_te_freq_continuum(mode, lengths, eps_r: float = 1.0) -> float:
    """Continuum PEC-box resonance f = v/2 sqrt(sum (m_i / L_i)^2)."""
    v = C0 / math.sqrt(eps_r)
    return 0.5 * v * math.sqrt(sum((m / L) ** 2 for m, L in zip(mode, lengths)))


def hybrid_modes(omega_p: float, delta: float, g: float):
    """Eq. omega_pm: omega_pm = omega_p + Delta/2 +- sqrt(Delta^2 + 4 g^2)/2."""
    r = 0.5 * math.sqrt(delta * delta + 4 * g * g)
    return omega_p + 0.5 * delta - r, omega_p + 0.5 * delta + r
