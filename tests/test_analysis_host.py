"""Interfacial analysis through the C ABI (ising_analysis.cpp) against the
oracle's numpy restatement on the same inputs: agreement to 1e-12 relative
(both reduce the same FP64 numbers; only the summation order differs), plus
the error statuses of bad arguments."""
import math

import numpy as np
import pytest

import paper_1411_5588_gb300 as ig
from oracle import analysis as OA
from paper_1411_5588_gb300 import analysis as A

REL = 1e-12


def close(a, b, scale=None):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    s = np.maximum(np.abs(b), 1.0 if scale is None else scale)
    return bool(np.all(np.abs(a - b) <= REL * s))


@pytest.fixture(scope="module")
def rng():
    return np.random.default_rng(20141120)


def test_layer_profile_and_mirror(rng):
    Lx, Ly, Lz = 7, 10, 12
    recs = np.zeros((50, 5 + Lx), dtype=np.int64)
    recs[:, 5:] = rng.integers(-Ly * Lz, Ly * Lz + 1, size=(50, Lx))
    recs[:, 0] = np.arange(50)
    for first in (0, 13, 49):
        assert close(A.layer_profile(recs, Lx, Ly, Lz, first), OA.layer_profile(recs, Lx, Ly, Lz, first))
    m = rng.normal(size=Lx)
    assert np.array_equal(A.mirror_profile(m), OA.mirror_profile(m))


def test_layer_profile_sums_are_exact_beyond_2_53():
    """Large layer sums over many records stay exact (int128 on the product
    side, Python integers in the oracle)."""
    Lx, Ly, Lz = 2, 1 << 15, 1 << 15
    recs = np.zeros((4, 5 + Lx), dtype=np.int64)
    recs[:, 5] = (1 << 30) - 1
    recs[:, 6] = -(1 << 30) + 3
    assert close(A.layer_profile(recs, Lx, Ly, Lz), OA.layer_profile(recs, Lx, Ly, Lz))


@pytest.mark.parametrize("k", [(1, None), (3, 18)])
def test_contact_angle(rng, k):
    Lx, Ly = 20, 80
    kx = np.arange(1, Lx + 1)
    mp = 0.9 + 0.01 * rng.normal(size=Lx)
    mm = -0.9 + 0.01 * rng.normal(size=Lx)
    y = 40 + 0.7 * (kx - 10) + rng.normal(size=Lx)
    mbar = (y * mp + (Ly - y) * mm) / Ly
    k_hi = Lx if k[1] is None else k[1]
    tg, yg = A.contact_angle(Ly, mbar, mp, mm, k[0], k_hi)
    to, yo = OA.contact_angle(Ly, mbar, mp, mm, k[0], k_hi)
    assert close(tg, to) and close(yg, yo, scale=Ly)


def test_young_difference_and_angle(rng):
    for n in (1, 4, 16, 33):
        m1, mn = rng.uniform(0.2, 1, n), rng.uniform(0.2, 1, n)
        assert close(A.ti_young_difference(0.55, m1, mn), OA.ti_young_difference(0.55, m1, mn))
    for d in (-0.7, -0.1, 0.0, 0.3):
        assert close(A.young_angle(d, 0.9), OA.young_angle(d, 0.9))


def test_gamma_of_theta(rng):
    th = np.sort(rng.uniform(0.3, math.pi / 2, 40))[::-1].copy()
    th[0] = math.pi / 2
    d = 0.8 * np.cos(th) + 0.01 * rng.normal(size=th.size)
    assert close(A.gamma_of_theta(th, d, 0.84), OA.gamma_of_theta(th, d, 0.84))


def test_free_energy_beta(rng):
    b = np.linspace(0.2, 0.9, 57)
    U = rng.normal(size=b.size) * 10
    for F0 in (0.0, -3.5):
        assert close(A.ti_free_energy_beta(b, U, F0), OA.ti_free_energy_beta(b, U, F0), scale=10.0)
    bd = b[::-1].copy()
    assert close(A.ti_free_energy_beta(bd, U, 2.0), OA.ti_free_energy_beta(bd, U, 2.0), scale=10.0)


def test_eq20_and_line_tension(rng):
    Lx = np.array([20.0, 26, 32, 40, 50])
    Lz = Lx.copy()
    dF = Lz * Lx * 0.7 - 0.4 * Lz + rng.normal(size=5)
    assert close(A.fit_gamma_tau(Lx, Lz, dF), OA.fit_gamma_tau(Lx, Lz, dF))
    args = (812.5, 48, 288, 96, 1.05, 0.93, 0.88, -0.031, -0.29)
    assert close(A.line_tension_residual(*args), OA.line_tension_residual(*args), scale=812.5)
    Lzs = np.array([16.0, 32, 48, 64, 96])
    R = -0.3 * Lzs + rng.normal(size=5)
    assert close(A.line_tension_lz_scan(Lzs, R), OA.line_tension_lz_scan(Lzs, R))


def test_stiffness_step_and_roughening(rng):
    th = math.pi / 2 - np.linspace(-0.3, 0.3, 13)
    g = 0.9 * (1 + 0.4 * (math.pi / 2 - th) ** 2) + 1e-3 * rng.normal(size=13)
    assert close(A.stiffness(th, g, 0.9), OA.stiffness(th, g, 0.9))
    th = math.pi / 2 - np.linspace(0.01, 0.1, 8)
    g = 1.5 + 0.6 * (math.pi / 2 - th) + 1e-3 * rng.normal(size=8)
    assert close(A.step_free_energy(th, g), OA.step_free_energy(th, g))
    phis = np.linspace(0.01, 0.1, 4)
    th = np.concatenate([math.pi / 2 - phis, math.pi / 2 + phis])  # both sides of pi/2
    g = 1.5 + 0.6 * np.abs(math.pi / 2 - th) + 1e-3 * rng.normal(size=8)
    assert close(A.step_free_energy(th, g), OA.step_free_energy(th, g))
    T = np.array([2.5, 2.6, 2.7, 3.0])
    k = T * (math.pi / 2) * (1 - 1.5 * np.sqrt((T - 2.45) / 4.51)) + 1e-3 * rng.normal(size=4)
    assert close(A.roughening_kappa_fit(T, k, 2.45, 4.51), OA.roughening_kappa_fit(T, k, 2.45, 4.51))
    T = np.array([1.0, 1.4, 1.8, 2.2])
    fs = 2 * np.exp(-0.7 / np.sqrt(1 - T / 2.45)) * (1 + 0.01 * rng.normal(size=4))
    assert close(A.roughening_fs_fit(T, fs, 2.45), OA.roughening_fs_fit(T, fs, 2.45))


def test_step_model_matches_and_never_overflows():
    for H1 in (0.0, 0.2, 0.45, 0.9):
        for Lz in (8, 16, 40):
            assert close(A.step_model(H1, 1.1, 1.5, 32, Lz), OA.step_model(H1, 1.1, 1.5, 32, Lz))
    # Lz / T large: the written-out weights overflow, the product's do not
    phi, hs = A.step_model(3.0, 1.0, 0.5, 64, 5000)
    assert phi == pytest.approx(1 / 64, rel=1e-15) and math.isfinite(hs)
    with pytest.raises(OverflowError):
        OA.step_model(3.0, 1.0, 0.5, 64, 5000)


def test_bad_arguments_are_einval():
    bad = [
        lambda: A.layer_profile(np.zeros((0, 7), dtype=np.int64), 2, 2, 2),
        lambda: A.contact_angle(10, [0.1, 0.2], [1, 1], [1, -1]),  # m+ = m- in layer 1
        lambda: A.contact_angle(10, [0.1, 0.2, 0.3], [1, 1, 1], [-1, -1, -1], 2, 2),
        lambda: A.young_angle(1.5, 1.0),
        lambda: A.gamma_of_theta([0.0, 1.0], [0.1, 0.1], 1.0),
        lambda: A.ti_free_energy_beta([0.0, 0.3], [1.0, 2.0]),
        lambda: A.fit_gamma_tau([20, 20], [20, 30], [1.0, 2.0]),
        lambda: A.line_tension_lz_scan([16, 16], [0.1, 0.2]),
        lambda: A.stiffness([math.pi / 2], [1.0], 1.0),
        lambda: A.roughening_kappa_fit([2.0], [1.0], 2.45, 4.51),
        lambda: A.roughening_fs_fit([2.5, 2.6], [1.0, 1.0], 2.45),
        lambda: A.step_model(0.1, 1.0, 0.0, 32, 16),
    ]
    for f in bad:
        with pytest.raises(ig.IsingError) as e:
            f()
        assert e.value.status == ig.EINVAL


def test_critical_field(rng):
    H1 = np.linspace(0.05, 0.8, 31)
    tilt = np.where(H1 < 0.4, 1e-4 * rng.random(31), (H1 - 0.4) * 0.9)
    theta = math.pi / 2 - tilt
    a = A.critical_field(H1, theta, 0.01, 2.0, 64, 128)
    b = OA.critical_field(H1, theta, 0.01, 2.0, 64, 128)
    assert close(a, b)
    for bad in ((H1, np.full(31, math.pi / 2)), (H1[::-1].copy(), theta)):
        with pytest.raises(ig.IsingError):
            A.critical_field(bad[0], bad[1], 0.01, 2.0, 64, 128)
