"""Analytic frame and speed-up relations of Sec. 2 (test infrastructure only).

Plain restatements of Vay et al. (arXiv:1009.2727), Sec. 2 and Sec. 5.1.1, in
SI units with CODATA 2018 constants. Used by the oracle's pin tests only.
"""
from __future__ import annotations

import math

C = 299792458.0
QE = 1.602176634e-19
ME = 9.1093837015e-31
EPS0 = 8.8541878128e-12


def omega_p(n_e: float) -> float:
    """Plasma frequency sqrt(n e^2/(eps0 m_e)) (Sec. 2, after the beta_w equation)."""
    return math.sqrt(n_e * QE * QE / (EPS0 * ME))


def lambda_p(n_e: float) -> float:
    """Wake wavelength lambda_p ~ 2 pi c/omega_p (Sec. 2)."""
    return 2.0 * math.pi * C / omega_p(n_e)


def beta_wake(n_e: float, lam: float) -> float:
    """Wake group velocity beta_w = (1 + omega_p^2/omega^2)^(-1/2) (Sec. 2, first equation)."""
    om = 2.0 * math.pi * C / lam
    return (1.0 + omega_p(n_e) ** 2 / om ** 2) ** -0.5


def gamma_wake(n_e: float, lam: float) -> float:
    """Relativistic factor of the wake, 1/sqrt(1 - beta_w^2) (= sqrt(1 + omega^2/omega_p^2))."""
    b = beta_wake(n_e, lam)
    return 1.0 / math.sqrt(1.0 - b * b)


def dephasing_length(n_e: float, lam: float) -> float:
    """L_d = lambda_p^3/(2 lambda^2) (Sec. 2)."""
    return lambda_p(n_e) ** 3 / (2.0 * lam * lam)


def boosted(gamma: float, n_e: float, lam: float, L: float, eta: float) -> dict:
    """Quantities in a frame moving at beta c (Sec. 2, boosted-frame block)."""
    beta = math.sqrt(1.0 - 1.0 / (gamma * gamma))
    bw = beta_wake(n_e, lam)
    lp = lambda_p(n_e)
    lp_s = lp / (gamma * (1.0 - bw * beta))
    L_s = L / gamma
    lam_s = gamma * (1.0 + beta) * lam
    bw_s = (bw - beta) / (1.0 - bw * beta)
    T_s = (L_s + eta * lp_s) / ((bw_s + beta) * C)
    R_s = T_s * C / lam_s
    return dict(beta=beta, lambda_p=lp_s, L=L_s, lam=lam_s, beta_w=bw_s, T=T_s, R=R_s)


def r_lab(n_e: float, lam: float, L: float, eta: float) -> float:
    """Cost in laser periods in the laboratory, R_lab = (L + eta lambda_p)/(beta_w lambda) (Sec. 2)."""
    return (L + eta * lambda_p(n_e)) / (beta_wake(n_e, lam) * lam)


def speedup_exact(gamma: float, n_e: float, lam: float, L: float, eta: float) -> float:
    """Eq. Eq_scaling1d0: S = (1+beta)(L + eta lambda_p)/((1 - beta beta_w) L + eta lambda_p)."""
    beta = math.sqrt(1.0 - 1.0 / (gamma * gamma))
    bw = beta_wake(n_e, lam)
    lp = lambda_p(n_e)
    return (1.0 + beta) * (L + eta * lp) / ((1.0 - beta * bw) * L + eta * lp)


def speedup_approx(gamma: float, gamma_w: float, xi: float, eta: float) -> float:
    """Eq. Eq_scaling1d (gamma_w^2 >> 1, L = xi L_d)."""
    beta = math.sqrt(1.0 - 1.0 / (gamma * gamma))
    num = xi * gamma_w ** 2
    return (1.0 + beta) ** 2 * gamma ** 2 * num / (num + (1.0 + beta) * gamma ** 2 * (xi * beta / 2.0 + 2.0 * eta))


def speedup_gamma_inf(gamma_w: float, xi: float, eta: float) -> float:
    """Eq. Eq_scaling_gamma_inf: 4 gamma_w^2/(1 + 4 eta/xi)."""
    return 4.0 / (1.0 + 4.0 * eta / xi) * gamma_w ** 2


def speedup_wake_frame(gamma_w: float, xi: float, eta: float) -> float:
    """Eq. Eq_scaling_gamma_wake: 2 gamma_w^2/(1 + 2 eta/xi)."""
    return 2.0 / (1.0 + 2.0 * eta / xi) * gamma_w ** 2


def boosted_dz(gamma: float, dz_lab: float) -> float:
    """Longitudinal cell kept at a fixed fraction of the laser wavelength: dz* = (1+beta) gamma dz (Sec. 5.1.1)."""
    beta = math.sqrt(1.0 - 1.0 / (gamma * gamma))
    return (1.0 + beta) * gamma * dz_lab


def speedup_yee_2d(S: float, dx: float, dz: float, dz_s: float) -> float:
    """Eq. Eq_scaling2d: Yee-CFL-limited 2D speed-up."""
    return S * dz * math.sqrt(1 / dx ** 2 + 1 / dz ** 2) / (dz_s * math.sqrt(1 / dx ** 2 + 1 / dz_s ** 2))


def laser_amplitude_ratio(gamma: float) -> float:
    """E'0/E0 = omega'/omega = 1/((1+beta) gamma) (Sec. 3.1.2)."""
    beta = math.sqrt(1.0 - 1.0 / (gamma * gamma))
    return 1.0 / ((1.0 + beta) * gamma)
