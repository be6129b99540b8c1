"""Interfacial analysis of the paper's Secs. II B-IV (host FP64, C ABI).

Argument marshalling only: every formula runs in the library
(``ising_analysis.cpp``).  Angles are in radians, energies in units of J.
"""
from __future__ import annotations

import ctypes as _c

import numpy as np

from .binding import _ptr, check, lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _out():
    return _c.c_double()


def layer_profile(records, Lx, Ly, Lz, first=0):
    """Eq. 17: per-site layer magnetisations averaged over records[first:]."""
    r = np.ascontiguousarray(records, dtype=np.int64)
    if r.ndim != 2 or r.shape[1] != 5 + Lx:
        raise ValueError("records must be (n, 5 + Lx)")
    out = np.zeros(Lx)
    check(lib().ising_layer_profile(_ptr(r), r.shape[0], int(Lx), int(Ly), int(Lz), int(first), _ptr(out)),
          "ising_layer_profile")
    return out


def mirror_profile(m_plus):
    """Eq. 12: the (-) profile from the (+) one."""
    mp = _f64(m_plus)
    out = np.zeros_like(mp)
    check(lib().ising_mirror_profile(mp.size, _ptr(mp), _ptr(out)), "ising_mirror_profile")
    return out


def contact_angle(Ly, mbar, m_plus, m_minus, k_lo=1, k_hi=None):
    """Eq. 18 and the dividing plane: returns (theta, y_plus)."""
    mb, mp, mm = _f64(mbar), _f64(m_plus), _f64(m_minus)
    Lx = mb.size
    k_hi = Lx if k_hi is None else k_hi
    y = np.zeros(Lx)
    th = _out()
    check(lib().ising_contact_angle(Lx, int(Ly), _ptr(mb), _ptr(mp), _ptr(mm), int(k_lo), int(k_hi), _ptr(y),
                                    _c.byref(th)), "ising_contact_angle")
    return th.value, y


def ti_young_difference(H1, m1, mn):
    """Eq. 9 over Gauss-Legendre nodes on [0, H1]."""
    a, b = _f64(m1), _f64(mn)
    out = _out()
    check(lib().ising_ti_young_difference(a.size, float(H1), _ptr(a), _ptr(b), _c.byref(out)),
          "ising_ti_young_difference")
    return out.value


def young_angle(delta_f1, gamma_pi2):
    """Eq. 8 (acute angle)."""
    out = _out()
    check(lib().ising_young_angle(float(delta_f1), float(gamma_pi2), _c.byref(out)), "ising_young_angle")
    return out.value


def gamma_of_theta(theta, delta_f1, gamma0):
    """Eq. 16 integrated from gamma(theta[0]) = gamma0."""
    t, d = _f64(theta), _f64(delta_f1)
    out = np.zeros_like(t)
    check(lib().ising_gamma_of_theta(t.size, _ptr(t), _ptr(d), float(gamma0), _ptr(out)), "ising_gamma_of_theta")
    return out


def ti_free_energy_beta(beta, U, F0=0.0):
    """Eq. 19 along beta from F(beta[0]) = F0."""
    b, u = _f64(beta), _f64(U)
    out = np.zeros_like(b)
    check(lib().ising_ti_free_energy_beta(b.size, _ptr(b), _ptr(u), float(F0), _ptr(out)),
          "ising_ti_free_energy_beta")
    return out


def fit_gamma_tau(Lx, Lz, dF):
    """Eq. 20: returns (gamma(pi/2), tau(0, pi/2))."""
    x, z, f = _f64(Lx), _f64(Lz), _f64(dF)
    g, t = _out(), _out()
    check(lib().ising_fit_gamma_tau(x.size, _ptr(x), _ptr(z), _ptr(f), _c.byref(g), _c.byref(t)),
          "ising_fit_gamma_tau")
    return g.value, t.value


def line_tension_residual(dF_film, Lx, Ly, Lz, theta, gamma_theta, gamma_pi2, s_wall, delta_f1):
    """Eq. 21 solved for 2 Lz [tau(H1, theta) - tau(0, pi/2)]."""
    out = _out()
    args = [float(v) for v in (dF_film, Lx, Ly, Lz, theta, gamma_theta, gamma_pi2, s_wall, delta_f1)]
    check(lib().ising_line_tension_residual(*args, _c.byref(out)), "ising_line_tension_residual")
    return out.value


def line_tension_lz_scan(Lz, R):
    """Constant-area size scan: returns (dtau, intercept)."""
    z, r = _f64(Lz), _f64(R)
    d, a = _out(), _out()
    check(lib().ising_line_tension_lz_scan(z.size, _ptr(z), _ptr(r), _c.byref(d), _c.byref(a)),
          "ising_line_tension_lz_scan")
    return d.value, a.value


def stiffness(theta, gamma, gamma_pi2):
    """Eqs. 23-24: returns (c, kappa)."""
    t, g = _f64(theta), _f64(gamma)
    c, k = _out(), _out()
    check(lib().ising_stiffness(t.size, _ptr(t), _ptr(g), float(gamma_pi2), _c.byref(c), _c.byref(k)),
          "ising_stiffness")
    return c.value, k.value


def roughening_kappa_fit(T, kappa, T_R, T_c):
    """Eq. 25: returns C."""
    t, k = _f64(T), _f64(kappa)
    out = _out()
    check(lib().ising_roughening_kappa_fit(t.size, _ptr(t), _ptr(k), float(T_R), float(T_c), _c.byref(out)),
          "ising_roughening_kappa_fit")
    return out.value


def step_free_energy(theta, gamma):
    """Eq. 26: returns (f_s, gamma_flat)."""
    t, g = _f64(theta), _f64(gamma)
    f, a = _out(), _out()
    check(lib().ising_step_free_energy(t.size, _ptr(t), _ptr(g), _c.byref(f), _c.byref(a)),
          "ising_step_free_energy")
    return f.value, a.value


def roughening_fs_fit(T, f_s, T_R):
    """Eq. 27: returns (A, log_amp)."""
    t, f = _f64(T), _f64(f_s)
    A, a = _out(), _out()
    check(lib().ising_roughening_fs_fit(t.size, _ptr(t), _ptr(f), float(T_R), _c.byref(A), _c.byref(a)),
          "ising_roughening_fs_fit")
    return A.value, a.value


def critical_field(H1, theta, tol, T, Lx, Lz):
    """Sec. III C and Eq. 32: returns (H1*, f_s)."""
    h, t = _f64(H1), _f64(theta)
    a, b = _out(), _out()
    check(lib().ising_critical_field(h.size, _ptr(h), _ptr(t), float(tol), float(T), float(Lx), float(Lz),
                                     _c.byref(a), _c.byref(b)), "ising_critical_field")
    return a.value, b.value


def step_model(H1, f_s, T, Lx, Lz):
    """Eqs. 28-32: returns (phi, h1_star)."""
    p, h = _out(), _out()
    check(lib().ising_step_model(float(H1), float(f_s), float(T), float(Lx), float(Lz), _c.byref(p), _c.byref(h)),
          "ising_step_model")
    return p.value, h.value
