"""Host FP64 integration (Eqs. 9, 19): product C functions vs the oracle's
numpy restatement, and both against closed forms."""
import math

import numpy as np
import pytest

import paper_1411_5588_gb300 as ig
from oracle import ti as OT


@pytest.mark.parametrize("a,b", [(0.0, 0.75), (0.3, 1.1), (-1.0, 2.0)])
@pytest.mark.parametrize("n", [1, 2, 5, 16, 33])
def test_gauss_legendre_exact_for_polynomials(n, a, b):
    """n nodes integrate every polynomial of degree <= 2n-1 exactly, on
    intervals that start at 0 and elsewhere."""
    for x, w in (ig.gauss_legendre(n, a, b), OT.gauss_legendre(n, a, b)):
        assert abs(w.sum() - (b - a)) < 1e-14
        assert np.allclose(x, (a + b) - x[::-1], atol=1e-15)  # symmetric about the midpoint
        for deg in range(0, 2 * n):
            exact = (b ** (deg + 1) - a ** (deg + 1)) / (deg + 1)
            got = float(np.sum(w * x ** deg))
            assert abs(got - exact) <= 1e-13 * max(1.0, abs(exact))


def test_product_and_oracle_nodes_agree():
    x1, w1 = ig.gauss_legendre(16, 0.0, 0.75)
    x2, w2 = OT.gauss_legendre(16, 0.0, 0.75)
    assert np.allclose(x1, x2, rtol=1e-14, atol=1e-15)
    assert np.allclose(w1, w2, rtol=1e-13, atol=1e-15)


def test_surface_field_integral_closed_form():
    """m1 - mn = 0.3 - 0.2 H1 + 0.05 H1^3 integrates exactly with 16 nodes."""
    H1 = 0.55
    x, _ = ig.gauss_legendre(16, 0.0, H1)
    diff = 0.3 - 0.2 * x + 0.05 * x ** 3
    m1, mn = 0.5 * diff + 0.1, -0.5 * diff + 0.1
    exact = -(0.3 * H1 - 0.1 * H1 ** 2 + 0.0125 * H1 ** 4)
    a = ig.ti_surface_field(H1, m1, mn)
    b = OT.surface_field_ti(H1, m1, mn)
    assert abs(a - exact) < 1e-14 and abs(b - exact) < 1e-14
    assert abs(a - b) <= 1e-12 * abs(b)


def test_trapezoids():
    T = np.linspace(1.5, 4.4, 40)
    U = -3.0 + 0.4 * T
    beta = 1.0 / T
    for got in (ig.ti_beta_trapezoid(beta, U), OT.beta_trapezoid(beta, U)):
        want = float(np.sum(0.5 * np.diff(beta) * (U[1:] + U[:-1])))
        assert abs(got - want) < 1e-13
    a = ig.ti_temperature_trapezoid(T, U)
    b = OT.temperature_trapezoid(T, U)
    assert abs(a - b) <= 1e-12 * abs(b)
    # refinement converges to the exact integral of (-3 + 0.4 T) d(1/T)
    # -integral_{1.5}^{4.4} (-3/T^2 + 0.4/T) dT = -[3/T + 0.4 ln T]
    exact = -((3.0 / 4.4 - 3.0 / 1.5) + 0.4 * math.log(4.4 / 1.5))
    Tf = np.linspace(1.5, 4.4, 20001)
    assert abs(ig.ti_temperature_trapezoid(Tf, -3.0 + 0.4 * Tf) - exact) < 1e-7


def test_series_mean_is_exact():
    big = np.array([[2 ** 62, 1], [2 ** 62, 2], [2 ** 62, 4], [3, 8]], dtype=np.int64)
    want = (3 * 2 ** 62 + 3) / 4
    assert ig.series_mean(big, 0) == want
    assert OT.series_mean(big, 0) == want
    assert ig.series_mean(big, 1, first=1) == 14 / 3


def test_series_energy_matches_the_oracle_film_energy():
    """Eq. 1 from the records (product C, exact integer column sums) against
    the oracle's own energy of the lattice after every sweep, and the mean
    against the oracle's numpy restatement."""
    from oracle import oracle as O
    for ym, H, H1 in ((O.Y_GAPBC, 0.0, 0.55), (O.Y_PBC, 0.1, -0.3), (O.Y_APBC, -0.2, 0.0)):
        f = O.Film(5, 6, 10, 1.3, H1, 2.7, 4, y_mode=ym, H=H)
        f.init(O.INIT_RANDOM)
        recs, want = [], []
        for _ in range(12):
            recs.append(f.sweep(1, 1)[0])
            want.append(f.energy())
        recs = np.array(recs)
        E, mean = ig.series_energy(recs, 1.3, H1, H=H, first=2)
        assert np.allclose(E, want, rtol=1e-14, atol=1e-12)
        m = OT.series_energy_mean(recs, 1.3, H, H1, 2)
        assert abs(mean - m) <= 1e-12 * max(1.0, abs(m))
        assert abs(mean - np.mean(want[2:])) <= 1e-12 * max(1.0, abs(m))
