"""Pins of the oracle's interfacial analysis (oracle/analysis.py) to what the
paper and the mathematics fix: exact enumeration of tiny films, Kaufman's
closed form for the 2D torus, the T = 0 limits the paper states, lattice
configurations of known geometry, and closed-form inputs.  A dropped term,
a wrong sign, a reversed index or a swapped argument in any function fails
one of these."""
import math

import numpy as np
import pytest

import exact as X
from oracle import analysis as OA
from oracle import oracle as O
from oracle import ti as OT

KAUFMAN_PATTERN = {"pbc": (1, 1, 1, 1), "apbc": (1, 1, -1, -1)}


def _binned(x, nbins=40):
    x = np.asarray(x, dtype=np.float64)
    b = x[: len(x) // nbins * nbins].reshape(nbins, -1).mean(axis=1)
    return float(b.mean()), float(b.std(ddof=1) / math.sqrt(nbins))


# ----------------------------------------------------------- Eqs. 12, 17

def test_layer_profile_is_the_per_site_layer_mean():
    """Eq. 17 on the oracle's own records of a fixed lattice: the mean over
    layer kx of the spins, with the record's m(kx) columns and Ly Lz."""
    Lx, Ly, Lz = 5, 6, 8
    rng = np.random.default_rng(3)
    recs = []
    want = np.zeros(Lx)
    for _ in range(4):
        s = rng.choice(np.array([-1, 1], dtype=np.int8), Lx * Ly * Lz, p=[0.3, 0.7])
        f = O.Film(Lx, Ly, Lz, 1.0, 0.4, 3.0, 1)
        f.set_spins(s)
        recs.append(f.measure())
        want += s.reshape(Lx, Ly, Lz).mean(axis=(1, 2)) / 4
    got = OA.layer_profile(np.array(recs), Lx, Ly, Lz)
    assert np.allclose(got, want, rtol=0, atol=1e-15)
    got2 = OA.layer_profile(np.array(recs), Lx, Ly, Lz, first=3)
    assert np.allclose(got2, s.reshape(Lx, Ly, Lz).mean(axis=(1, 2)), rtol=0, atol=1e-15)


def test_mirror_profile_matches_the_minus_phase_of_the_oracle():
    """Eq. 12 as a property of the simulated ensemble: a periodic-y film at
    T = 3 started all up stays in (+), started all down stays in (-), and
    <m(-)(kx)> = -<m(+)(Lx + 1 - kx)> within sampling error.  Without the
    reversal the walls' fields (+-H1) make the profiles differ."""
    Lx, Ly, Lz, H1, T = 6, 8, 8, 0.6, 3.0
    prof = {}
    for sign in (1, -1):
        f = O.Film(Lx, Ly, Lz, 1.0, H1, T, 11, y_mode=O.Y_PBC, replica=1 if sign > 0 else 2)
        f.set_spins(np.full(Lx * Ly * Lz, sign, dtype=np.int8))
        f.sweep(200)
        r = f.sweep(4000, 1)
        prof[sign] = [_binned(r[:, 5 + k] / (Ly * Lz)) for k in range(Lx)]
    m_plus = np.array([p[0] for p in prof[1]])
    m_minus = np.array([p[0] for p in prof[-1]])
    err = np.array([p[1] for p in prof[1]])[::-1] + np.array([p[1] for p in prof[-1]])
    pred = OA.mirror_profile(m_plus)
    assert np.all(np.abs(pred - m_minus) < 5 * err + 1e-12)
    # without the reversal (m- = -m+ layer by layer) the walls' fields show
    err_flat = np.array([p[1] for p in prof[1]]) + err - np.array([p[1] for p in prof[1]])[::-1]
    assert np.any(np.abs(-m_plus - m_minus) > 10 * err_flat)


# ---------------------------------------------------------------- Eq. 18

def test_contact_angle_recovers_a_synthetic_plane():
    """mbar built from Eq. 18 with y+(kx) on a plane of known angle and
    arbitrary layer plateaus gives back y+ and the angle."""
    Lx, Ly = 20, 64
    kx = np.arange(1, Lx + 1)
    for theta0 in (math.pi / 2, 1.2, math.pi / 4, 0.4):
        y_plus = 30.0 + (kx - 10.5) / math.tan(theta0) * (-1 if theta0 < 1 else 1)
        mp = 0.9 - 0.2 * np.exp(-(kx - 1)) + 0.1 * np.exp(-(Lx - kx))
        mm = -0.85 + 0.05 * np.sin(kx)
        mbar = (y_plus * mp + (Ly - y_plus) * mm) / Ly
        th, y = OA.contact_angle(Ly, mbar, mp, mm)
        assert np.allclose(y, y_plus, rtol=0, atol=1e-11)
        assert abs(th - theta0) < 1e-12


@pytest.mark.parametrize("theta0", [math.pi / 3, math.radians(75), math.radians(40)])
def test_contact_angle_of_a_lattice_staircase(theta0):
    """A real configuration: in layer kx the rows ky <= round(yc + (kx - c)
    cot(theta0)) are up, the rest down.  Its record from the oracle's own
    measurement, with m+ = +1 and m- = -1, gives y+ exactly equal to the
    row counts and theta within the staircase rounding."""
    Lx, Ly, Lz = 24, 64, 4
    cot = 1.0 / math.tan(theta0)
    rows = np.array([int(round(32 + (k - 12.5) * cot)) for k in range(1, Lx + 1)])
    s = -np.ones((Lx, Ly, Lz), dtype=np.int8)
    for k in range(Lx):
        s[k, : rows[k], :] = 1
    f = O.Film(Lx, Ly, Lz, 1.0, 0.3, 3.0, 1)
    f.set_spins(s.reshape(-1))
    mbar = OA.layer_profile(f.measure()[None, :], Lx, Ly, Lz)
    th, y = OA.contact_angle(Ly, mbar, np.ones(Lx), -np.ones(Lx))
    assert np.allclose(y, rows, rtol=0, atol=1e-12)
    assert abs(th - theta0) < 0.01


# ------------------------------------------------------------ Eqs. 8, 9

def test_young_difference_is_exact_for_polynomials():
    """Gauss-Legendre on [0, H1] integrates m1 + mn of degree <= 2n - 1
    exactly, and it is m1 + mn (not m1 - mn) that enters."""
    H1, n = 0.7, 8
    t, _ = np.polynomial.legendre.leggauss(n)
    x = 0.5 * H1 * (t + 1)
    m1 = 0.9 + 0.1 * x - 0.3 * x ** 5
    mn = 0.4 - 0.2 * x ** 2 + x ** 15 * 0.01
    exact = -(0.9 * H1 + 0.05 * H1 ** 2 - 0.05 * H1 ** 6 + 0.4 * H1 - 0.2 / 3 * H1 ** 3 + 0.01 / 16 * H1 ** 16)
    assert abs(OA.ti_young_difference(H1, m1, mn) - exact) < 1e-14


def test_young_difference_at_low_temperature_is_twice_the_field():
    """Eqs. 4, 7, 9 at T -> 0: in a (+) film both wall layers are saturated
    (m1 = mn = 1), so the Young difference f1(+)(H1) - f1(-)(H1) is the
    surface energy difference -2 H1; the film's own integral over H1
    (m1 - mn, Eq. 21's wall term) vanishes there.  Oracle films at T = 1."""
    Lx, Ly, Lz, T, H1, n = 4, 4, 8, 1.0, 0.5, 4
    t, _ = np.polynomial.legendre.leggauss(n)
    nodes = 0.5 * H1 * (t + 1)
    m1, mn = [], []
    for i, h in enumerate(nodes):
        f = O.Film(Lx, Ly, Lz, 1.0, float(h), T, 21, y_mode=O.Y_PBC, replica=i)
        f.init(O.INIT_ALL_UP)
        r = f.sweep(400, 1)
        m1.append(r[:, 3].mean() / (Ly * Lz))
        mn.append(r[:, 4].mean() / (Ly * Lz))
    d = OA.ti_young_difference(H1, m1, mn)
    assert abs(d - (-2 * H1)) < 5e-3
    assert abs(OT.surface_field_ti(H1, m1, mn)) < 5e-3
    # Eq. 8 at T = 0: gamma(pi/2) = 2J, so cos(theta) = H1 / J
    assert abs(OA.young_angle(-2 * H1, 2.0) - math.acos(H1)) < 1e-15


def test_film_integral_over_h1_is_the_exact_free_energy_change():
    """The film's own integral over its surface field, -int <M1 - Mn> dH1
    (Eq. 1 with Hn = -H1), equals F(H1) - F(0) = -T ln Z(H1)/Z(0) from
    exact enumeration of a 12-spin film with the Eq. 11 boundary."""
    Lx, Ly, Lz, T, H1 = 2, 3, 2, 3.0, 0.6
    N = Lx * Ly * Lz
    S = X.configs_pm1(N)
    bonds = X.bond_list(Lx, Ly, Lz, X.Y_GAPBC)
    B, M, m = X.observables(S, Lx, Ly, Lz, bonds)

    def E(h):
        return -B - h * m[:, 0] + h * m[:, Lx - 1]

    def logZ(h):
        e = -E(h) / T
        top = e.max()
        return top + math.log(np.exp(e - top).sum())

    t, _ = np.polynomial.legendre.leggauss(16)
    nodes = 0.5 * H1 * (t + 1)
    M1, Mn = [], []
    for h in nodes:
        w = np.exp(-(E(h) - E(h).min()) / T)
        w /= w.sum()
        M1.append(float((w * m[:, 0]).sum()))
        Mn.append(float((w * m[:, Lx - 1]).sum()))
    got = OT.surface_field_ti(H1, M1, Mn)
    want = -T * (logZ(H1) - logZ(0.0))
    assert abs(got - want) < 1e-11 * abs(want)


# ---------------------------------------------------------------- Eq. 16

def _theta_grid(n):
    return np.linspace(math.pi / 2, math.pi / 6, n)


def test_gamma_of_theta_isotropic_tension():
    """delta_f1 = gamma0 cos(theta) (plain Young) gives back a constant
    tension, to the trapezoid rule's O(h^2)."""
    for n, tol in ((201, 2e-5), (401, 5e-6)):
        th = _theta_grid(n)
        g = OA.gamma_of_theta(th, 1.3 * np.cos(th), 1.3)
        assert np.max(np.abs(g - 1.3)) < tol


def test_gamma_of_theta_zero_temperature_shape():
    """T = 0: gamma(theta) = gamma0 (sin + cos) (two broken bonds per unit
    step, Sec. III A) satisfies Eq. 16 with the constant delta_f1 = gamma0;
    integrating back gives it, with gamma(pi/4) = sqrt(2) gamma(pi/2), and
    the error falls by 4 when the step halves."""
    errs = []
    for n in (101, 201, 401):
        th = np.linspace(math.pi / 2, math.pi / 4, n)
        g = OA.gamma_of_theta(th, np.full(n, 2.0), 2.0)
        want = 2.0 * (np.sin(th) + np.cos(th))
        errs.append(np.max(np.abs(g - want)))
        assert abs(g[-1] / g[0] - math.sqrt(2)) < 1e-3
    assert 3.6 < errs[0] / errs[1] < 4.4 and 3.6 < errs[1] / errs[2] < 4.4


# ---------------------------------------------------------------- Eq. 19

def test_free_energy_by_beta_integration_matches_enumeration():
    """Eq. 19 for U = U_APBC - U_PBC of a 16-spin film (free x, H1 = 0):
    from beta0 = 0.2 with the exact dF(beta0), the trapezoid rule reaches
    the exact F_APBC - F_PBC = -T ln(Z_A / Z_P) at every point."""
    Lx, Ly, Lz = 2, 4, 2
    S = X.configs_pm1(Lx * Ly * Lz)
    Es = {}
    for name, mode in (("A", X.Y_APBC), ("P", X.Y_PBC)):
        Es[name] = X.energies(S, Lx, Ly, Lz, 1.0, 0.0, 0.0, mode).astype(np.float64)

    def logZ(E, b):
        e = -b * E
        top = e.max()
        return top + math.log(np.exp(e - top).sum())

    def U(E, b):
        w = np.exp(-b * (E - E.min()))
        return float((w * E).sum() / w.sum())

    beta = np.linspace(0.2, 1.2, 2001)
    dU = np.array([U(Es["A"], b) - U(Es["P"], b) for b in beta])
    exact = np.array([-(logZ(Es["A"], b) - logZ(Es["P"], b)) / b for b in beta])
    F = OA.ti_free_energy_beta(beta, dU, exact[0])
    assert np.max(np.abs(F - exact)) < 1e-6 * np.max(np.abs(exact))
    # a start deep in the ordered phase, downwards in beta
    bd = np.linspace(6.0, 0.5, 4001)
    dUd = np.array([U(Es["A"], b) - U(Es["P"], b) for b in bd])
    exd = np.array([-(logZ(Es["A"], b) - logZ(Es["P"], b)) / b for b in bd])
    Fd = OA.ti_free_energy_beta(bd, dUd, exd[0])
    assert np.max(np.abs(Fd - exd)) < 1e-5 * np.max(np.abs(exd))


def test_interface_free_energy_of_the_2d_torus_by_beta_integration():
    """Lx = 1 films are 2D tori: U_A - U_P from Kaufman's closed form
    (antiperiodic vs periodic y), integrated over beta from 0.2, gives
    Kaufman's -T ln(Z_A / Z_P) on a 16 x 16 torus through T_c, with the
    trapezoid rule's h^2 convergence; at beta = 0.6 dF / L is within a few
    percent of Onsager's tension 2J + T ln tanh(beta J).  (Beyond beta ~ 0.6
    Z_A is a difference of nearly equal products, and its numerical
    derivative loses the digits this check needs.)"""
    L = 16

    def logZ(b, p):
        return X.kaufman_logZ(b, L, L, KAUFMAN_PATTERN[p])

    def U(b, p):
        return -X.kaufman_energy_per_bond_sum(b, L, L, KAUFMAN_PATTERN[p])

    errs = []
    for n in (601, 1201):
        beta = np.linspace(0.2, 0.6, n)
        dU = np.array([U(b, "apbc") - U(b, "pbc") for b in beta])
        exact = np.array([-(logZ(b, "apbc") - logZ(b, "pbc")) / b for b in beta])
        F = OA.ti_free_energy_beta(beta, dU, exact[0])
        errs.append(np.max(np.abs(F - exact)))
    assert errs[1] < 2e-6 * abs(exact[-1])
    assert 3.5 < errs[0] / errs[1] < 4.5
    sigma = 2.0 + math.log(math.tanh(0.6)) / 0.6
    assert abs(F[-1] / L - sigma) < 0.05 * sigma


# ------------------------------------------------------------- Eqs. 20-22

def test_fit_gamma_tau_recovers_the_line_term():
    Lx = np.array([20.0, 30.0, 40.0, 50.0])
    Lz = Lx.copy()
    dF = Lz * Lx * 0.73 + 2 * Lz * (-0.21)
    g, t = OA.fit_gamma_tau(Lx, Lz, dF)
    assert abs(g - 0.73) < 1e-13 and abs(t + 0.21) < 1e-12


def test_line_tension_residual_and_scan_on_the_constant_area_set():
    """Eq. 21 assembled from known terms on the constant-area set of
    Sec. II C (Lx Lz = 4608, Ly Lz = 27648): the residual is 2 Lz dtau and
    the scan returns dtau with a zero intercept; a missing area term would
    leave Lz-independent offsets only if areas are constant, so a second
    set with varying areas must fail the straight line."""
    gamma_pi2, theta, gamma_theta, s_wall, df1, dtau = 0.9, 1.1, 0.95, -0.03, -0.4, -0.17
    R = []
    sizes = [(96, 576, 48), (48, 288, 96), (24, 144, 192)]
    for Lx, Ly, Lz in sizes:
        dF = (Lx * Lz * (gamma_theta / math.sin(theta) - gamma_pi2) + Lz * Ly * s_wall
              + Lz * Lx * df1 / math.tan(theta) + 2 * Lz * dtau)
        r = OA.line_tension_residual(dF, Lx, Ly, Lz, theta, gamma_theta, gamma_pi2, s_wall, df1)
        assert abs(r - 2 * Lz * dtau) < 1e-9
        R.append(r)
    d, a = OA.line_tension_lz_scan([s[2] for s in sizes], R)
    assert abs(d - dtau) < 1e-13 and abs(a) < 1e-10


# ------------------------------------------------------------- Eqs. 23-27

def test_stiffness_of_an_exact_quadratic_and_of_gamma_plus_second_derivative():
    """Eq. 23 data give c exactly; for gamma = g0 (1 + c cos^2 theta),
    Eq. 24's gamma(pi/2) + gamma''(pi/2) (finite differences) equals the
    fitted kappa to O(phi^2)."""
    th = math.pi / 2 - np.linspace(-0.2, 0.2, 21)
    g = 1.1 * (1 + 0.35 * (math.pi / 2 - th) ** 2)
    c, k = OA.stiffness(th, g, 1.1)
    assert abs(c - 0.35) < 1e-13 and abs(k - 1.1 * 1.7) < 1e-13

    def gam(t):
        return 1.1 * (1 + 0.35 * math.cos(t) ** 2)

    h = 1e-4
    kappa_fd = gam(math.pi / 2) + (gam(math.pi / 2 + h) - 2 * gam(math.pi / 2) + gam(math.pi / 2 - h)) / h ** 2
    th = math.pi / 2 - np.linspace(-0.05, 0.05, 11)
    c2, k2 = OA.stiffness(th, [gam(t) for t in th], gam(math.pi / 2))
    assert abs(k2 - kappa_fd) < 1e-3


def test_roughening_fits_recover_their_constants():
    Tc, TR = 4.5115, 2.45
    T = np.array([2.55, 2.6, 2.65, 3.0])
    kappa = T * (math.pi / 2) * (1 - 1.57 * np.sqrt((T - TR) / Tc))
    assert abs(OA.roughening_kappa_fit(T, kappa, TR, Tc) - 1.57) < 1e-13
    Tl = np.array([1.0, 1.5, 2.0, 2.3])
    fs = 3.0 * np.exp(-0.8 * (1 - Tl / TR) ** -0.5)
    A, la = OA.roughening_fs_fit(Tl, fs, TR)
    assert abs(A - 0.8) < 1e-12 and abs(la - math.log(3.0)) < 1e-12


def test_step_free_energy_at_zero_temperature():
    """The T = 0 tension gamma0 (sin + cos) has |dgamma/dtheta| = gamma0 at
    pi/2 (a unit step costs 2J per unit length, gamma0 = 2J)."""
    phi = np.linspace(0.002, 0.02, 10)
    th = math.pi / 2 - phi
    g = 2.0 * (np.sin(th) + np.cos(th))
    fs, g0 = OA.step_free_energy(th, g)
    assert abs(fs - 2.0) < 0.03 and abs(g0 - 2.0) < 1e-3


def test_step_free_energy_on_both_sides_of_the_cusp():
    """Eq. 26 takes the tilt's magnitude: a tilt either way from pi/2 costs
    the same, so the T = 0 tension gamma0 (|sin| + |cos|) sampled on both
    sides of the flat orientation still gives f_s = gamma0."""
    phi = np.linspace(0.002, 0.02, 10)
    th = np.concatenate([math.pi / 2 - phi, math.pi / 2 + phi])
    g = 2.0 * (np.abs(np.sin(th)) + np.abs(np.cos(th)))
    fs, g0 = OA.step_free_energy(th, g)
    assert abs(fs - 2.0) < 0.03 and abs(g0 - 2.0) < 1e-3


def test_step_model_limits():
    """Eqs. 28-32: no tilt at H1 = 0; at H1 = H1* the up-step weight equals
    the flat one (which defines Eq. 32); a strong field saturates at one
    step over Lx, phi -> 1/Lx."""
    fs, T, Lx, Lz = 1.2, 1.0, 32, 24
    phi, hs = OA.step_model(0.0, fs, T, Lx, Lz)
    assert phi == 0.0
    assert abs(hs - (0.6 - math.log(32) / 48)) < 1e-15
    phi, _ = OA.step_model(hs, fs, T, Lx, Lz)
    Wm = Lx * math.exp(-fs * Lz / T - 2 * hs * Lz / T)
    assert abs(phi - (1 - Wm) / (2 + Wm) / Lx) < 1e-15
    phi, _ = OA.step_model(1.0, fs, T, Lx, Lz)
    assert abs(phi - 1 / Lx) < 1e-6 / Lx


def test_critical_field_recovers_the_step_model_onset():
    """Sec. III C: theta(H1) drawn from the single-step model (Eqs. 28-31)
    with a known f_s; at H1* of Eq. 32 the up-step weight equals the flat
    one, so the tilt there is (1 - W-1)/((2 + W-1) Lx), and the crossing of
    that tilt gives back H1* and f_s (to the scan's resolution)."""
    fs, T, Lx, Lz = 1.1, 1.5, 48, 64
    hs = 0.5 * fs - T * math.log(Lx) / (2 * Lz)
    Wm = Lx * math.exp(-fs * Lz / T - 2 * hs * Lz / T)
    tol = (1 - Wm) / (2 + Wm) / Lx
    H1 = np.linspace(0.0, 0.6, 2401)
    theta = np.array([math.pi / 2 - OA.step_model(h, fs, T, Lx, Lz)[0] for h in H1])
    h, f = OA.critical_field(H1, theta, tol, T, Lx, Lz)
    assert abs(h - hs) < 1e-4 and abs(f - fs) < 2e-4
