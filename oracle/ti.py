"""Thermodynamic-integration arithmetic of the paper -- TEST INFRASTRUCTURE ONLY.

Plain numpy restatement, independent of the product's C implementation:
  The film's own integral over H1: with Hn = -H1 written into Eq. 1,
         dF/dH1 = -<M1> + <Mn>, so F(H1) - F(0) = -integral_0^{H1}
         (m_1 - m_n) dH1'.  In a uniform film this is the wall term of Eq. 21;
         the Young difference of Eq. 9 (m_1 + m_n) is in oracle/analysis.py.
  Eq. 19 (Sec. II C): beta F(beta) - beta0 F(beta0) = integral U dbeta, by the
         trapezoid rule in beta, or over T as -integral U / T^2 dT.
Gauss-Legendre nodes come from numpy's library routine.
"""
from __future__ import annotations

import numpy as np


def gauss_legendre(n, a, b):
    t, w = np.polynomial.legendre.leggauss(int(n))
    half, mid = 0.5 * (b - a), 0.5 * (b + a)
    return mid + half * t, half * w


def series_mean(records, col, first=0):
    """Exact integer mean of one record column (Python integers, one division)."""
    vals = [int(v) for v in np.asarray(records)[first:, col]]
    return float(sum(vals)) / len(vals) if len(vals) < 2 ** 53 else sum(vals) / len(vals)


def series_energy_mean(records, J, H, H1, first=0):
    """Eq. 1 averaged over records[first:], from exact (Python integer)
    column sums: -J <B> - H <M> - H1 <M1> - Hn <Mn>, Hn = -H1."""
    r = np.asarray(records)[first:]
    n = len(r)
    B, M, M1, Mn = (sum(int(v) for v in r[:, c]) / n for c in (1, 2, 3, 4))
    return -J * B - H * M - H1 * M1 + H1 * Mn


def surface_field_ti(H1, m1, mn):
    """-integral_0^{H1} (m1 - mn) over Gauss-Legendre nodes on [0, H1]."""
    x, w = gauss_legendre(len(m1), 0.0, H1)
    return -float(np.sum(w * (np.asarray(m1, dtype=np.float64) - np.asarray(mn, dtype=np.float64))))


def beta_trapezoid(beta, U):
    b = np.asarray(beta, dtype=np.float64)
    u = np.asarray(U, dtype=np.float64)
    return float(np.sum(0.5 * (b[1:] - b[:-1]) * (u[1:] + u[:-1])))


def temperature_trapezoid(T, U):
    t = np.asarray(T, dtype=np.float64)
    g = np.asarray(U, dtype=np.float64) / t ** 2
    return -float(np.sum(0.5 * (t[1:] - t[:-1]) * (g[1:] + g[:-1])))
