"""Interfacial analysis of Secs. II B-IV -- TEST INFRASTRUCTURE ONLY.

Plain numpy restatement of the paper's post-processing, independent of the
product's C implementation (it shares no code with it and calls only numpy).
Each function follows one passage:

  Eq. 12   m^(-)(kx) = -m^(+)(Lx + 1 - kx)
  Eq. 17   mbar_kx, the per-site layer magnetisation, averaged over records
  Eq. 18   Ly mbar = y+ m+ + y- m-, y+ + y- = Ly; the dividing plane and theta
  Eq. 9    delta_f1 = -int_0^{H1} (m_1 + m_n) dH1'  (Young difference; by
           Eqs. 4 and 7 it is f1(+)(H1) - f1(-)(H1))
  Eq. 8    f_int cos(theta) = delta_f1
  Eq. 16   gamma cos(theta) - gamma' sin(theta) = delta_f1, as
           d(gamma / sin)/dtheta = -delta_f1 / sin^2, trapezoid over the points
  Eq. 19   beta F(beta) - beta0 F(beta0) = int U dbeta, trapezoid
  Eq. 20   dF / (Lz Lx) = gamma(pi/2) + (2 / Lx) tau(0, pi/2)
  Eq. 21   solved for 2 Lz [tau(H1, theta) - tau(0, pi/2)]
  Eqs. 23-25, 26-27, 28-32  stiffness, roughening fits, step model
  Sec. III C              the critical field H1* and f_s from Eq. 32

Fits use numpy's least-squares routine (``np.linalg.lstsq``) as a library
step.  Every function is pinned in tests/test_oracle_analysis.py (closed
forms, exact enumeration, Kaufman's torus, the T = 0 limits, the step
model), so none is parity-unpinned.
"""
from __future__ import annotations

import math

import numpy as np


def _lsq(columns, y):
    A = np.stack([np.asarray(c, dtype=np.float64) for c in columns], axis=1)
    coef, *_ = np.linalg.lstsq(A, np.asarray(y, dtype=np.float64), rcond=None)
    return coef


def mirror_profile(m_plus):
    """Eq. 12."""
    return -np.asarray(m_plus, dtype=np.float64)[::-1].copy()


def layer_profile(records, Lx, Ly, Lz, first=0):
    """Eq. 17 from the m(kx) columns (Python integers, one division)."""
    r = np.asarray(records)[first:]
    out = np.empty(Lx)
    for k in range(Lx):
        total = sum(int(v) for v in r[:, 5 + k])
        out[k] = total / (len(r) * Ly * Lz)
    return out


def contact_angle(Ly, mbar, m_plus, m_minus, k_lo=1, k_hi=None):
    """Eq. 18 per layer, then the plane y+(kx) = a + b kx; theta = atan(1/|b|)."""
    mbar, mp, mm = (np.asarray(v, dtype=np.float64) for v in (mbar, m_plus, m_minus))
    Lx = len(mbar)
    k_hi = Lx if k_hi is None else k_hi
    y_plus = Ly * (mbar - mm) / (mp - mm)
    kx = np.arange(k_lo, k_hi + 1, dtype=np.float64)
    a, b = _lsq([np.ones_like(kx), kx], y_plus[k_lo - 1:k_hi])
    return math.atan2(1.0, abs(b)), y_plus


def ti_young_difference(H1, m1, mn):
    """Eq. 9 on Gauss-Legendre nodes of [0, H1] (numpy's nodes)."""
    t, w = np.polynomial.legendre.leggauss(len(m1))
    w = 0.5 * H1 * w
    return -float(np.sum(w * (np.asarray(m1, dtype=np.float64) + np.asarray(mn, dtype=np.float64))))


def young_angle(delta_f1, gamma_pi2):
    """Eq. 8, acute angle."""
    return math.acos(abs(delta_f1) / gamma_pi2)


def gamma_of_theta(theta, delta_f1, gamma0):
    """Eq. 16 integrated from gamma(theta[0]) = gamma0."""
    th = np.asarray(theta, dtype=np.float64)
    rhs = -np.asarray(delta_f1, dtype=np.float64) / np.sin(th) ** 2
    steps = 0.5 * np.diff(th) * (rhs[1:] + rhs[:-1])
    g = gamma0 / math.sin(th[0]) + np.concatenate([[0.0], np.cumsum(steps)])
    out = g * np.sin(th)
    out[0] = gamma0
    return out


def ti_free_energy_beta(beta, U, F0=0.0):
    """Eq. 19 along beta from F(beta[0]) = F0."""
    b = np.asarray(beta, dtype=np.float64)
    u = np.asarray(U, dtype=np.float64)
    steps = 0.5 * np.diff(b) * (u[1:] + u[:-1])
    bF = b[0] * F0 + np.concatenate([[0.0], np.cumsum(steps)])
    out = bF / b
    out[0] = F0
    return out


def fit_gamma_tau(Lx, Lz, dF):
    """Eq. 20."""
    Lx, Lz, dF = (np.asarray(v, dtype=np.float64) for v in (Lx, Lz, dF))
    gamma, tau = _lsq([np.ones_like(Lx), 2.0 / Lx], dF / (Lz * Lx))
    return float(gamma), float(tau)


def line_tension_residual(dF_film, Lx, Ly, Lz, theta, gamma_theta, gamma_pi2, s_wall, delta_f1):
    """Eq. 21: what is left of F_int(H1) - F_int(0) after the area terms."""
    area_tilt = Lx * Lz * (gamma_theta / math.sin(theta) - gamma_pi2)
    walls = Lz * Ly * s_wall + Lz * Lx * delta_f1 / math.tan(theta)
    return dF_film - area_tilt - walls


def line_tension_lz_scan(Lz, R):
    """Constant-area scan: R = intercept + 2 Lz dtau."""
    Lz = np.asarray(Lz, dtype=np.float64)
    intercept, slope = _lsq([np.ones_like(Lz), Lz], R)
    return 0.5 * float(slope), float(intercept)


def stiffness(theta, gamma, gamma_pi2):
    """Eqs. 23-24."""
    phi2 = (math.pi / 2 - np.asarray(theta, dtype=np.float64)) ** 2
    (c,) = _lsq([phi2], np.asarray(gamma, dtype=np.float64) / gamma_pi2 - 1.0)
    return float(c), gamma_pi2 * (1.0 + 2.0 * float(c))


def roughening_kappa_fit(T, kappa, T_R, T_c):
    """Eq. 25: kappa beta = (pi/2) [1 - C ((T - T_R)/T_c)^(1/2)]."""
    T = np.asarray(T, dtype=np.float64)
    y = 1.0 - np.asarray(kappa, dtype=np.float64) / T / (math.pi / 2)
    (C,) = _lsq([np.sqrt((T - T_R) / T_c)], y)
    return float(C)


def step_free_energy(theta, gamma):
    """Eq. 26 as the slope of gamma against |pi/2 - theta|."""
    phi = np.abs(math.pi / 2 - np.asarray(theta, dtype=np.float64))
    gamma_flat, slope = _lsq([np.ones_like(phi), phi], gamma)
    return abs(float(slope)), float(gamma_flat)


def roughening_fs_fit(T, f_s, T_R):
    """Eq. 27 with f_s ~ 1/xi_R: ln f_s = ln a - A (1 - T/T_R)^(-1/2)."""
    x = (1.0 - np.asarray(T, dtype=np.float64) / T_R) ** -0.5
    log_amp, slope = _lsq([np.ones_like(x), x], np.log(np.asarray(f_s, dtype=np.float64)))
    return -float(slope), float(log_amp)


def critical_field(H1, theta, tol, T, Lx, Lz):
    """Sec. III C: the tilt pi/2 - theta first exceeds tol between two scan
    points; H1* is where their straight line crosses tol.  Eq. 32 solved for
    f_s gives f_s = 2 H1* + T ln(Lx) / Lz."""
    H1 = np.asarray(H1, dtype=np.float64)
    tilt = math.pi / 2 - np.asarray(theta, dtype=np.float64)
    above = np.nonzero(tilt > tol)[0]
    i = int(above[0])
    if i == 0:
        raise ValueError("tilt above tol at the first point")
    h = H1[i - 1] + (tol - tilt[i - 1]) * (H1[i] - H1[i - 1]) / (tilt[i] - tilt[i - 1])
    return float(h), 2.0 * float(h) + T * math.log(Lx) / Lz


def step_model(H1, f_s, T, Lx, Lz):
    """Eqs. 28-32 with the weights written out (Python floats; moderate
    arguments only, large exponents overflow here by design)."""
    W0 = 1.0
    Wp = Lx * math.exp(-f_s * Lz / T) * math.exp(2 * H1 * Lz / T)
    Wm = Lx * math.exp(-f_s * Lz / T) * math.exp(-2 * H1 * Lz / T)
    Z = W0 + Wp + Wm
    phi = (Wp - Wm) / Z / Lx
    h1_star = 0.5 * f_s - T * math.log(Lx) / (2 * Lz)
    return phi, h1_star
