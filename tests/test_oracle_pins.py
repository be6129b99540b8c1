"""Pins of the oracle against what the paper and the mathematics fix.

Each test checks ``oracle/`` against something other than itself: published
Philox known-answer vectors and an independent library implementation,
brute-force enumeration of tiny films, the exact transition matrix of the
sweep, exact symmetries of Eq. 1 with the boundary rules of Sec. II A, the
T -> 0 and beta = 0 limits, and Kaufman's closed form for the 2D torus that a
one-layer film reduces to.
"""
import ctypes
import ctypes.util
import math
import os

import numpy as np
import pytest

import exact as X
from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ Philox

def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(t, 16) for t in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers():
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = O.philox4x32_10([ctr], key)[0]
        assert [int(v) for v in got] == want


def _curand():
    for name in ("libcurand.so", "libcurand.so.10"):
        for d in ("/usr/local/cuda/lib64", "/usr/local/cuda/targets/sbsa-linux/lib",
                  "/usr/local/cuda/targets/x86_64-linux/lib", ""):
            try:
                return ctypes.CDLL(os.path.join(d, name) if d else name)
            except OSError:
                continue
    return None


@pytest.mark.parametrize("seed", [0x0000000500000007, 0xDEADBEEFCAFEF00D, 1])
def test_philox_matches_curand_host_generator(seed):
    """curand's host Philox4_32_10 generator emits block b of four words as
    Philox4x32-10(ctr = (b >> 16, 0, b & 0xFFFF, 0), key = (lo32 seed, hi32 seed))."""
    cu = _curand()
    if cu is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    assert cu.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # CURAND_RNG_PSEUDO_PHILOX4_32_10
    try:
        assert cu.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        nblk = 70000
        buf = np.zeros(4 * nblk, dtype=np.uint32)
        assert cu.curandGenerate(gen, buf.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(buf.size)) == 0
    finally:
        cu.curandDestroyGenerator(gen)
    b = np.arange(nblk, dtype=np.uint64)
    ctr = np.zeros((nblk, 4), dtype=np.uint32)
    ctr[:, 0] = (b >> 16).astype(np.uint32)
    ctr[:, 2] = (b & 0xFFFF).astype(np.uint32)
    out = O.philox4x32_10(ctr, [seed & 0xFFFFFFFF, seed >> 32])
    assert np.array_equal(out.reshape(-1), buf)


# --------------------------------------------------- energy and measurement

def _random_film(Lx, Ly, Lz, H1, T, y_mode, seed, H=0.0, x_mode=O.X_FREE):
    f = O.Film(Lx, Ly, Lz, 1.0, H1, T, seed, y_mode=y_mode, x_mode=x_mode, H=H)
    f.init(O.INIT_RANDOM)
    return f


@pytest.mark.parametrize("shape", [(5, 6, 4), (4, 4, 2), (3, 2, 6), (1, 3, 4), (6, 5, 8)])
@pytest.mark.parametrize("y_mode", [O.Y_GAPBC, O.Y_PBC, O.Y_APBC])
def test_record_matches_independent_bond_list(shape, y_mode):
    Lx, Ly, Lz = shape
    f = _random_film(Lx, Ly, Lz, 0.3, 3.0, y_mode, seed=11)
    f.sweep(3)
    s = f.get_spins()
    rec = f.measure()
    bonds = X.bond_list(Lx, Ly, Lz, y_mode)
    B, M, m = X.observables(s[None, :], Lx, Ly, Lz, bonds)
    assert rec[0] == 3
    assert rec[1] == B[0]
    assert rec[2] == M[0]
    assert rec[3] == m[0, 0] and rec[4] == m[0, Lx - 1]
    assert np.array_equal(rec[5:], m[0])


@pytest.mark.parametrize("y_mode", [O.Y_GAPBC, O.Y_PBC, O.Y_APBC])
@pytest.mark.parametrize("x_mode", [O.X_FREE, O.X_PBC])
def test_delta_e_is_energy_difference(y_mode, x_mode):
    """dE of every site equals E(flipped) - E(original) from Eq. 1."""
    Lx, Ly, Lz, J, H, H1 = 4, 5, 6, 1.0, 0.17, 0.55
    f = O.Film(Lx, Ly, Lz, J, H1, 2.5, 5, y_mode=y_mode, x_mode=x_mode, H=H)
    f.init(O.INIT_RANDOM)
    s = f.get_spins().astype(np.int64)
    E0 = X.energies(s[None, :], Lx, Ly, Lz, J, H, H1, y_mode, x_mode == O.X_PBC)[0]
    for kx in range(1, Lx + 1):
        for ky in range(1, Ly + 1):
            for kz in range(1, Lz + 1):
                i = X.site_index(Lx, Ly, Lz, kx - 1, ky - 1, kz - 1)
                t = s.copy()
                t[i] = -t[i]
                E1 = X.energies(t[None, :], Lx, Ly, Lz, J, H, H1, y_mode, x_mode == O.X_PBC)[0]
                assert abs(f.delta_e(kx, ky, kz) - (E1 - E0)) < 1e-9


# ---------------------------------------------------- exact symmetries

@pytest.mark.parametrize("shape", [(5, 8, 6), (4, 6, 4), (3, 5, 2)])
def test_gapbc_translation_invariance(shape):
    """Sec. II A: with Eq. 11 the film is translation invariant along y.  The
    shift ky -> ky+1 whose wrapped row is S(Lx+1-kx, Ly) with its sign reversed
    leaves the Eq. 1 energy unchanged (H = 0)."""
    Lx, Ly, Lz = shape
    f = _random_film(Lx, Ly, Lz, 0.45, 3.0, O.Y_GAPBC, seed=3)
    f.sweep(2)
    s = f.get_spins().reshape(Lx, Ly, Lz)
    t = np.empty_like(s)
    t[:, 1:, :] = s[:, :-1, :]
    t[:, 0, :] = -s[::-1, Ly - 1, :]
    E = X.energies(np.stack([s.reshape(-1), t.reshape(-1)]), Lx, Ly, Lz, 1.0, 0.0, 0.45)
    assert abs(E[0] - E[1]) < 1e-9
    g = O.Film(Lx, Ly, Lz, 1.0, 0.45, 3.0, 1)
    g.set_spins(t.reshape(-1))
    assert abs(g.energy() - f.energy()) < 1e-9


@pytest.mark.parametrize("shape", [(5, 8, 6), (4, 6, 4)])
def test_reflection_symmetry_of_energy(shape):
    """Eq. 12: S(kx) -> -S(Lx+1-kx) maps the film onto itself (H = 0)."""
    Lx, Ly, Lz = shape
    f = _random_film(Lx, Ly, Lz, 0.45, 3.0, O.Y_GAPBC, seed=4)
    s = f.get_spins().reshape(Lx, Ly, Lz)
    r = -s[::-1, :, :]
    g = O.Film(Lx, Ly, Lz, 1.0, 0.45, 3.0, 1)
    g.set_spins(r.reshape(-1))
    assert abs(g.energy() - f.energy()) < 1e-9


@pytest.mark.parametrize("y_mode", [O.Y_GAPBC, O.Y_PBC, O.Y_APBC])
def test_spin_and_field_reversal_trajectory(y_mode):
    """Eqs. 3-6: reversing all spins together with H and H1 leaves every dE,
    hence every Metropolis decision, unchanged; trajectories are exact mirror
    images sweep by sweep."""
    Lx, Ly, Lz = 6, 8, 10
    a = O.Film(Lx, Ly, Lz, 1.0, 0.55, 2.7, 9, y_mode=y_mode, H=0.05)
    b = O.Film(Lx, Ly, Lz, 1.0, -0.55, 2.7, 9, y_mode=y_mode, H=-0.05)
    a.init(O.INIT_RANDOM)
    b.set_spins(-a.get_spins())
    ra = a.sweep(20, 1)
    rb = b.sweep(20, 1)
    assert np.array_equal(a.get_spins(), -b.get_spins())
    assert np.array_equal(ra[:, 1], rb[:, 1])
    assert np.array_equal(ra[:, 2:], -rb[:, 2:])


def test_beta_zero_negates_every_sweep():
    """beta = 0: exp(-dE/T) = 1, every attempted flip is accepted, so each
    sweep reverses every spin exactly."""
    f = O.Film(5, 6, 8, 1.0, 0.5, math.inf, 2)
    f.init(O.INIT_RANDOM)
    s0 = f.get_spins()
    f.sweep(1)
    assert np.array_equal(f.get_spins(), -s0)
    f.sweep(1)
    assert np.array_equal(f.get_spins(), s0)


def test_zero_temperature_never_raises_energy():
    """T -> 0: every dE > 0 threshold underflows to 0, only dE <= 0 moves are
    taken, so the Eq. 1 energy never increases."""
    f = O.Film(6, 8, 10, 1.0, 0.3, 1e-3, 7)
    f.init(O.INIT_RANDOM)
    e = [f.energy()]
    for _ in range(30):
        f.sweep(1)
        e.append(f.energy())
    assert all(e[i + 1] <= e[i] + 1e-12 for i in range(len(e) - 1))
    assert e[-1] < e[0]


@pytest.mark.parametrize("shape", [(2, 2, 4), (3, 2, 2), (2, 3, 2), (1, 4, 4), (3, 3, 2)])
def test_flat_interface_ground_state(shape):
    """With Eq. 11 and H1 = 0 the uniform state has every bond satisfied except
    the Lx*Lz wrap bonds, B = 3 LxLyLz - LyLz - 2 LxLz (bond counting, Sec.
    II C); enumeration confirms it is the maximum of B for Lx >= 2, and the
    oracle quenched from the uniform state at T -> 0 stays there."""
    Lx, Ly, Lz = shape
    want = 3 * Lx * Ly * Lz - Ly * Lz - 2 * Lx * Lz
    ex = X.exact_averages(Lx, Ly, Lz, 1.0, 0.0, 0.0, 1.0, X.Y_GAPBC)
    if Lx >= 2:
        assert ex["Bmax"] == want
    f = O.Film(Lx, Ly, Lz, 1.0, 0.0, 1e-3, 1)
    f.init(O.INIT_ALL_UP)
    assert f.measure()[1] == want
    f.sweep(5)
    assert f.measure()[1] == want


# ------------------------------------------------- RNG counter convention

def test_init_random_uses_init_counter():
    Lx, Ly, Lz = 3, 4, 20
    f = O.Film(Lx, Ly, Lz, 1.0, 0.0, 3.0, 0x1234_0000_5678)
    f.init(O.INIT_RANDOM)
    s = f.get_spins().reshape(Lx * Ly, Lz)
    key = [(0x5678 ^ 0x1234), 0]
    for row in range(Lx * Ly):
        for z0 in range(Lz):
            u = O.philox4x32_10([[row, z0 >> 3, 0xFFFFFFFF, 2 | (z0 & 1)]], key)[0][(z0 >> 1) & 3]
            assert s[row, z0] == (1 if u < 2 ** 31 else -1)


def test_sweep_counter_convention():
    """All-up periodic block at H = 0: every colour-0 site of the rows ky < Ly
    sees dE = 12 J in phase P0 and nothing later changes it, so after one sweep
    exactly the sites with u < floor(exp(-12/T) 2^32) are down, u being word
    (z0>>1)&3 of Philox(row, z0>>3, sweep, z0&1) under key (seed fold, replica)."""
    Lx, Ly, Lz, T = 4, 6, 16, 3.5
    f = O.Film(Lx, Ly, Lz, 1.0, 0.0, T, 77, y_mode=O.Y_PBC, x_mode=O.X_PBC, replica=5)
    f.init(O.INIT_ALL_UP)
    f.sweep_count = 123
    f.sweep(1)
    s = f.get_spins().reshape(Lx, Ly, Lz)
    thr = math.floor(math.ldexp(math.exp(-12.0 / T), 32))
    for kx in range(1, Lx + 1):
        for ky in range(1, Ly):
            for kz in range(1, Lz + 1):
                if (kx + ky + kz) % 2:
                    continue
                z0 = kz - 1
                row = (kx - 1) * Ly + (ky - 1)
                u = O.philox4x32_10([[row, z0 >> 3, 123, z0 & 1]], [77, 5])[0][(z0 >> 1) & 3]
                assert s[kx - 1, ky - 1, z0] == (-1 if u < thr else 1)


def test_acceptance_boundary_is_strict():
    """The Metropolis reading with a 32-bit word takes a move iff u <
    floor(exp(-dE/T) 2^32), so that it is accepted with probability exactly
    thr / 2^32: the word equal to the threshold is rejected and the one below
    it accepted (a chain could meet that word only once in 2^32 draws, so no
    statistical pin sees the difference); dE <= 0 is always accepted."""
    for dE, T in ((4.0, 3.0), (12.0, 2.2), (0.5, 0.7), (8.0, 1e-3 * 2 ** 10)):
        thr = math.floor(math.ldexp(math.exp(-dE / T), 32))
        assert 0 < thr < 2 ** 32
        assert O.accept(dE, T, thr - 1) and not O.accept(dE, T, thr)
    assert O.accept(0.0, 1.0, 0xFFFFFFFF) and O.accept(-4.0, 1.0, 0xFFFFFFFF)
    assert not O.accept(4.0, 1e-3, 0)  # exp(-4000) floors to a zero threshold


def test_records_fall_on_multiples_of_the_interval():
    """A record is taken after every completed sweep whose count is a
    multiple of the interval, the count running from 0 across calls (and from
    wherever it was set)."""
    f = O.Film(4, 6, 8, 1.0, 0.3, 3.0, 5)
    f.init(O.INIT_RANDOM)
    assert list(f.sweep(10, 3)[:, 0]) == [3, 6, 9]
    assert list(f.sweep(5, 3)[:, 0]) == [12, 15]
    f.sweep_count = 100
    assert list(f.sweep(7, 4)[:, 0]) == [104]
    assert list(f.sweep(2, 1)[:, 0]) == [108, 109]


# ------------------------------------------------------- transition matrix

def test_four_phase_schedule_preserves_boltzmann():
    """With exact Metropolis probabilities the four-phase sweep leaves the Eq. 1
    Boltzmann distribution invariant for every y mode, while the plain
    two-colour sweep does not once the Eq. 11 wrap joins equal colours
    (Lx + Ly even)."""
    args = dict(J=1.0, H=0.0, H1=0.4, T=2.0)
    for shape in [(2, 2, 2), (1, 5, 2), (1, 2, 4)]:
        for ym in (X.Y_GAPBC, X.Y_PBC, X.Y_APBC):
            P = X.transition_matrix(*shape, y_mode=ym, acc=X.exact_accept, **args)
            pi = X.boltzmann(*shape, args["J"], args["H"], args["H1"], args["T"], ym)
            assert np.allclose(pi @ P, pi, rtol=1e-12, atol=1e-15)
    P2 = X.transition_matrix(2, 2, 2, y_mode=X.Y_GAPBC, n_phases=2, acc=X.exact_accept, **args)
    pi = X.boltzmann(2, 2, 2, args["J"], args["H"], args["H1"], args["T"], X.Y_GAPBC)
    assert np.max(np.abs(pi @ P2 - pi) / pi) > 1e-3


def test_quantised_chain_stationary_close_to_boltzmann():
    P = X.transition_matrix(2, 2, 2, 1.0, 0.0, 0.5, 2.5)
    pi = X.boltzmann(2, 2, 2, 1.0, 0.0, 0.5, 2.5)
    st = X.stationary(P)
    assert np.max(np.abs(st - pi) / pi) < 1e-6


@pytest.mark.parametrize("y_mode", [O.Y_GAPBC, O.Y_PBC])
def test_one_sweep_distribution_matches_transition_matrix(y_mode):
    """The oracle's one-sweep move from a fixed state, repeated with many
    sweep counters (independent Philox streams), follows row s0 of the exact
    transition matrix (chi-square)."""
    Lx, Ly, Lz, H1, T = 2, 2, 2, 0.5, 2.2
    P = X.transition_matrix(Lx, Ly, Lz, 1.0, 0.0, H1, T, y_mode=y_mode)
    s0 = np.array([1, -1, 1, 1, -1, -1, 1, -1], dtype=np.int8)
    row = P[X.state_of(s0)]
    f = O.Film(Lx, Ly, Lz, 1.0, H1, T, 21, y_mode=y_mode)
    n = 40000
    counts = np.zeros(1 << 8)
    for t in range(n):
        f.set_spins(s0)
        f.sweep_count = t
        f.sweep(1)
        counts[X.state_of(f.get_spins())] += 1
    expected = row * n
    keep = expected > 5
    assert counts[~keep].sum() <= max(20, 3 * expected[~keep].sum() + 10)
    chi2 = float((((counts - expected) ** 2)[keep] / expected[keep]).sum())
    dof = int(keep.sum()) - 1
    # 5-sigma bound for chi-square with dof degrees of freedom
    assert chi2 < dof + 5 * math.sqrt(2 * dof)


# ---------------------------------------------- MC averages vs enumeration

def _binned_mean(x, nbins=50):
    x = np.asarray(x, dtype=np.float64)
    n = (x.size // nbins) * nbins
    b = x[:n].reshape(nbins, -1).mean(axis=1)
    return float(b.mean()), float(b.std(ddof=1) / math.sqrt(nbins))


CASES = [
    ((2, 2, 4), X.Y_GAPBC, 0.5, 3.0),
    ((2, 4, 2), X.Y_GAPBC, 1.0, 1.5),
    ((3, 2, 2), X.Y_APBC, 0.0, 4.5),
    ((3, 3, 2), X.Y_GAPBC, 0.5, 3.0),
    ((2, 3, 2), X.Y_GAPBC, 0.5, 1.5),
    ((1, 4, 4), X.Y_GAPBC, 0.5, 3.0),
    ((2, 2, 4), X.Y_PBC, 1.0, 3.0),
    ((3, 3, 2), X.Y_PBC, 0.5, 4.5),
]


@pytest.mark.parametrize("shape,y_mode,H1,T", CASES)
def test_mc_averages_match_enumeration(shape, y_mode, H1, T):
    Lx, Ly, Lz = shape
    ex = X.exact_averages(Lx, Ly, Lz, 1.0, 0.0, H1, T, y_mode)
    f = O.Film(Lx, Ly, Lz, 1.0, H1, T, 1234, y_mode=y_mode)
    f.init(O.INIT_RANDOM)
    f.sweep(1000)
    recs = f.sweep(200000, 1)
    E = -recs[:, 1] - H1 * recs[:, 3] + H1 * recs[:, 4]
    for name, series in (("E", E), ("M", recs[:, 2]), ("M1", recs[:, 3]), ("Mn", recs[:, 4]),
                         ("absM", np.abs(recs[:, 2]))):
        mu, err = _binned_mean(series)
        assert abs(mu - ex[name]) < 4 * err + 1e-9, (name, mu, ex[name], err)
    for k in range(Lx):
        mu, err = _binned_mean(recs[:, 5 + k])
        assert abs(mu - ex["m"][k]) < 4 * err + 1e-9


# ---------------------------------------------- one-layer film = 2D torus

KAUFMAN_PATTERN = {X.Y_PBC: (1, 1, 1, 1), X.Y_GAPBC: (1, 1, -1, -1)}


@pytest.mark.parametrize("y_mode", [X.Y_PBC, X.Y_GAPBC])
def test_kaufman_closed_form_matches_enumeration(y_mode):
    """Kaufman's m x n torus formula (m = Ly, n = Lz); with Lx = 1 the Eq. 11
    wrap is a plain antiperiodic y boundary, whose partition function takes
    the sign pattern (+,+,-,-) of the four products."""
    for Ly, Lz in [(4, 4), (3, 4), (5, 4), (2, 6)]:
        for T in (1.6, 2.269, 3.5):
            S = X.configs_pm1(Ly * Lz)
            E = X.energies(S, 1, Ly, Lz, 1.0, 0.0, 0.0, y_mode)
            logZ = float(np.log(np.exp(-E / T).sum()))
            got = X.kaufman_logZ(1.0 / T, Ly, Lz, KAUFMAN_PATTERN[y_mode])
            assert abs(got - logZ) < 1e-10 * abs(logZ)


@pytest.mark.parametrize("y_mode,L,T", [(X.Y_PBC, 16, 2.0), (X.Y_PBC, 16, 2.269), (X.Y_GAPBC, 16, 3.0),
                                        (X.Y_PBC, 32, 3.0)])
def test_one_layer_film_energy_matches_kaufman(y_mode, L, T):
    """Lx = 1: the +-H1 surface fields cancel on the single layer and the film
    is the 2D Ising torus; <B> from the oracle agrees with d log Z / dK."""
    want = X.kaufman_energy_per_bond_sum(1.0 / T, L, L, KAUFMAN_PATTERN[y_mode])
    f = O.Film(1, L, L, 1.0, 0.7, T, 99, y_mode=y_mode)
    f.init(O.INIT_RANDOM)
    f.sweep(2000)
    recs = f.sweep(60000, 1)
    mu, err = _binned_mean(recs[:, 1], nbins=40)
    assert abs(mu - want) < 4 * err, (mu, want, err)


# ------------------------------------------------------------ initial states

@pytest.mark.parametrize("p", [0.0, 0.01, 0.3, 1.0])
def test_slab_start_is_a_slab_with_binomial_flips(p):
    """SLAB_Y: +1 for ky <= Ly/2, -1 above, then each spin reversed with
    probability p -- the flip count is Binomial(N, floor(p 2^32)/2^32)."""
    Lx, Ly, Lz = 6, 11, 40
    f = O.Film(Lx, Ly, Lz, 1.0, 0.0, 3.0, 17)
    f.init(O.INIT_SLAB_Y, p)
    s = f.get_spins().reshape(Lx, Ly, Lz)
    slab = np.where(np.arange(1, Ly + 1) <= Ly // 2, 1, -1)[None, :, None]
    flipped = int((s != slab).sum())
    N = s.size
    q = math.floor(math.ldexp(p, 32)) / 2 ** 32
    if q in (0.0, 1.0):
        assert flipped == round(q * N)
    else:
        sd = math.sqrt(N * q * (1 - q))
        assert abs(flipped - N * q) < 5 * sd + 1


def test_random_start_is_balanced():
    f = O.Film(10, 12, 64, 1.0, 0.0, 3.0, 23)
    f.init(O.INIT_RANDOM)
    s = f.get_spins().astype(np.int64)
    assert abs(s.sum()) < 5 * math.sqrt(s.size)
