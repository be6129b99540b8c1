"""GPU path vs the CPU oracle, bit for bit (spins and int64 records).

Every case runs the same seeded chain on both sides -- same counter-based
Philox stream, same four-phase schedule, same binary64 thresholds -- so the
spin configuration and every record must be identical after any number of
sweeps.  Shapes cover several words per row with a ragged last word, a
single partial word, Lz = 2 (double z bonds), Ly = 2, Lx = 1, odd and even
Lx + Ly (the Eq. 11 wrap joining equal or opposite colours), periodic x,
thin films whose rows the one-word grid kernels pack two or four to a
register, and the degenerate temperatures beta = 0 and T -> 0.
"""
import math

import numpy as np
import pytest

import paper_1411_5588_gb300 as ig
from oracle import oracle as O

pytestmark = pytest.mark.gpu

#        Lx  Ly  Lz   y_mode      x_mode    H1     H    T      init            flip
CASES = [
    (8, 8, 8, ig.Y_GAPBC, ig.X_FREE, 0.5, 0.0, 3.0, ig.INIT_RANDOM, 0.0),
    (5, 6, 66, ig.Y_GAPBC, ig.X_FREE, 0.55, 0.0, 2.5, ig.INIT_RANDOM, 0.0),
    (3, 4, 2, ig.Y_GAPBC, ig.X_FREE, 0.3, 0.0, 2.0, ig.INIT_RANDOM, 0.0),
    (1, 8, 16, ig.Y_GAPBC, ig.X_FREE, 0.7, 0.0, 2.2, ig.INIT_RANDOM, 0.0),
    (4, 3, 130, ig.Y_PBC, ig.X_FREE, 0.2, 0.0, 3.5, ig.INIT_RANDOM, 0.0),
    (6, 2, 64, ig.Y_APBC, ig.X_FREE, 0.4, 0.0, 3.0, ig.INIT_RANDOM, 0.0),
    (7, 5, 128, ig.Y_GAPBC, ig.X_FREE, 0.45, 0.0, 3.0, ig.INIT_SLAB_Y, 0.01),
    (6, 5, 200, ig.Y_GAPBC, ig.X_FREE, 0.45, 0.0, 2.0, ig.INIT_SLAB_Y, 0.05),
    (4, 4, 8, ig.Y_PBC, ig.X_PBC, 0.0, 0.0, 4.5, ig.INIT_RANDOM, 0.0),
    (9, 10, 190, ig.Y_GAPBC, ig.X_FREE, -0.3, 0.1, 1.5, ig.INIT_SLAB_Y, 0.01),
    (5, 7, 64, ig.Y_GAPBC, ig.X_FREE, 0.5, 0.0, math.inf, ig.INIT_RANDOM, 0.0),
    (5, 7, 64, ig.Y_GAPBC, ig.X_FREE, 0.5, 0.0, 1e-3, ig.INIT_RANDOM, 0.0),
    (3, 3, 6, ig.Y_GAPBC, ig.X_FREE, 1.0, 0.0, 1.5, ig.INIT_ALL_UP, 0.0),
    (2, 9, 34, ig.Y_APBC, ig.X_PBC, 0.25, -0.2, 2.8, ig.INIT_RANDOM, 0.0),
    (16, 12, 96, ig.Y_GAPBC, ig.X_FREE, 0.55, 0.0, 3.0, ig.INIT_SLAB_Y, 0.01),
    # thin films, several rows per packed word in the one-word grid kernels
    (6, 12, 16, ig.Y_APBC, ig.X_FREE, 0.35, 0.0, 2.6, ig.INIT_RANDOM, 0.0),
    (5, 10, 30, ig.Y_GAPBC, ig.X_FREE, 0.45, 0.0, 3.0, ig.INIT_SLAB_Y, 0.02),
    (7, 16, 12, ig.Y_GAPBC, ig.X_FREE, -0.5, 0.0, 2.3, ig.INIT_SLAB_Y, 0.01),
    (4, 6, 20, ig.Y_PBC, ig.X_PBC, 0.0, 0.15, 3.4, ig.INIT_RANDOM, 0.0),
    (9, 8, 4, ig.Y_GAPBC, ig.X_FREE, 0.6, 0.0, 2.9, ig.INIT_RANDOM, 0.0),
    (6, 8, 16, ig.Y_GAPBC, ig.X_FREE, 0.5, 0.0, 1e-3, ig.INIT_RANDOM, 0.0),
]


def _pair(case, seed=7, replica=3, shape=ig.SHAPE_AUTO):
    Lx, Ly, Lz, ym, xm, H1, H, T, kind, flip = case
    g = ig.Film(Lx, Ly, Lz, 1.0, H1, T, seed, y_mode=ym, x_mode=xm, H=H, replica=replica, shape=shape)
    o = O.Film(Lx, Ly, Lz, 1.0, H1, T, seed, y_mode=ym, x_mode=xm, H=H, replica=replica)
    g.init(kind, flip)
    o.init(kind, flip)
    return g, o


SHAPES = [ig.SHAPE_RESIDENT, ig.SHAPE_GRID_1, ig.SHAPE_GRID_2, ig.SHAPE_GRID_Q, ig.SHAPE_CLUSTER]


@pytest.mark.parametrize("shape", SHAPES, ids=["resident", "grid1", "grid2", "gridq", "cluster"])
@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}x{c[1]}x{c[2]}-y{c[3]}x{c[4]}-T{c[7]}" for c in CASES])
def test_sweeps_bit_exact(case, shape):
    """Every launch shape: the resident kernel (the film in shared memory for
    the whole call), the grid kernels with one or two words per thread or
    four threads per word, and the cluster kernel (the film in the
    distributed shared memory of min(Lx, 8) CTAs for the whole call)."""
    g, o = _pair(case, shape=shape)
    assert np.array_equal(g.get_spins(), o.get_spins()), "initial state differs"
    done = 0
    for n, m in ((1, 1), (1, 1), (8, 2), (90, 3)):
        g.sweep(n, m)
        want = o.sweep(n, m)
        got = g.read_series()
        done += n
        assert g.sweep_count == done
        assert np.array_equal(got, want), f"records differ after {done} sweeps"
        assert np.array_equal(g.get_spins(), o.get_spins()), f"spins differ after {done} sweeps"
    assert np.array_equal(g.measure(), o.measure())
    g.close()


THIN = [  # films of at least 8192 rows that pack two rows per word (Lz 12, 30), and one that packs four
    (48, 172, 30, ig.Y_GAPBC, ig.X_FREE, 0.45, 0.0, 3.0, ig.INIT_SLAB_Y, 0.01),
    (64, 130, 12, ig.Y_APBC, ig.X_PBC, 0.0, 0.1, 2.7, ig.INIT_RANDOM, 0.0),
    (33, 256, 14, ig.Y_GAPBC, ig.X_FREE, -0.4, 0.0, 2.4, ig.INIT_RANDOM, 0.0),
    (40, 208, 16, ig.Y_PBC, ig.X_FREE, 0.3, 0.0, 3.2, ig.INIT_SLAB_Y, 0.02),
]


@pytest.mark.parametrize("case", THIN, ids=[f"{c[0]}x{c[1]}x{c[2]}-y{c[3]}" for c in THIN])
def test_large_thin_films_bit_exact(case):
    """Thin films large enough to pack two rows per word at one word per
    thread (and Lz = 16, four): the single-film kernel, then the same film in
    a batch beside a film that does not pack, with records every 1-3 sweeps
    (the summing launches take the rows one at a time)."""
    g, o = _pair(case, shape=ig.SHAPE_GRID_1)
    for n, m in ((1, 1), (6, 2), (21, 3)):
        g.sweep(n, m)
        assert np.array_equal(g.read_series(), o.sweep(n, m)), n
        assert np.array_equal(g.get_spins(), o.get_spins()), n
    g.close()
    Lx, Ly, Lz, ym, xm, H1, H, T, kind, flip = case
    specs = [dict(Lx=Lx, Ly=Ly, Lz=Lz, y_mode=ym, x_mode=xm, H1=H1, H=H, T=T, seed=7, replica=1, init_kind=kind,
                  flip_p=flip, measure_every=2),
             dict(Lx=6, Ly=9, Lz=70, T=2.5, H1=0.2, seed=7, replica=2, init_kind=ig.INIT_RANDOM, measure_every=1)]
    b = ig.Batch(specs, lanes=1)
    b.set_shape(ig.SHAPE_GRID_1)
    b.sweep(3, False)
    b.sweep(33, True)
    for i, sp in enumerate(specs):
        o = O.Film(sp["Lx"], sp["Ly"], sp["Lz"], 1.0, sp["H1"], sp["T"], sp["seed"], y_mode=sp.get("y_mode", 0),
                   x_mode=sp.get("x_mode", 0), H=sp.get("H", 0.0), replica=sp["replica"])
        o.init(sp["init_kind"], sp.get("flip_p", 0.0))
        assert np.array_equal(b.read_series(i), o.sweep(36, sp["measure_every"])), i
        assert np.array_equal(b.get_spins(i), o.get_spins()), i
    b.close()


def test_measure_matches_oracle_on_given_spins():
    rng = np.random.default_rng(5)
    for Lx, Ly, Lz, ym in [(5, 6, 66, ig.Y_GAPBC), (3, 4, 2, ig.Y_APBC), (6, 5, 200, ig.Y_PBC)]:
        s = np.where(rng.random(Lx * Ly * Lz) < 0.5, 1, -1).astype(np.int8)
        g = ig.Film(Lx, Ly, Lz, 1.0, 0.3, 2.0, 1, y_mode=ym)
        o = O.Film(Lx, Ly, Lz, 1.0, 0.3, 2.0, 1, y_mode=ym)
        g.set_spins(s)
        o.set_spins(s)
        assert np.array_equal(g.get_spins(), s)
        assert np.array_equal(g.measure(), o.measure())
        g.close()


def test_checkpoint_resume_is_bit_exact():
    case = (7, 6, 70, ig.Y_GAPBC, ig.X_FREE, 0.5, 0.0, 2.6, ig.INIT_RANDOM, 0.0)
    g, o = _pair(case, seed=11)
    g.sweep(37, 0)
    saved, at = g.get_spins(), g.sweep_count
    g.close()
    h = ig.Film(7, 6, 70, 1.0, 0.5, 2.6, 11, replica=3)
    h.set_spins(saved)
    h.sweep_count = at
    h.sweep(63, 7)
    rec = h.read_series()
    o.sweep(37, 0)
    want = o.sweep(63, 7)
    assert np.array_equal(rec, want)
    assert np.array_equal(h.get_spins(), o.get_spins())
    h.close()


@pytest.mark.parametrize("shape", SHAPES, ids=["resident", "grid1", "grid2", "gridq", "cluster"])
def test_sweeps_up_to_the_counter_limit_are_bit_exact(shape):
    """The sweep index is the third word of every Philox counter, and
    0xFFFFFFFF is reserved for the initial state's draws.  A film resumed 40
    sweeps before the limit runs 39 of them bit-exact (a record every 3
    sweeps, so the records' sweep column passes 2^32 - 2); the 40th sweep is
    refused before any device work, and the film carries on unchanged."""
    case = (9, 8, 70, ig.Y_GAPBC, ig.X_FREE, 0.45, 0.0, 3.0, ig.INIT_SLAB_Y, 0.1)
    g, o = _pair(case, seed=5, shape=shape)
    g.sweep(3, 0)
    o.sweep(3, 0)
    start = 0xFFFFFFFF - 40
    g.sweep_count = start
    o.sweep_count = start
    g.sweep(39, 3)
    want = o.sweep(39, 3)
    assert want[-1][0] == 0xFFFFFFFF - 1 - (0xFFFFFFFF - 1) % 3
    assert np.array_equal(g.read_series(), want)
    assert np.array_equal(g.get_spins(), o.get_spins())
    with pytest.raises(ig.IsingError) as e:
        g.sweep(1, 0)
    assert e.value.status == ig.EINVAL
    with pytest.raises(ValueError):
        o.sweep(1, 0)
    assert g.sweep_count == 0xFFFFFFFF - 1
    assert np.array_equal(g.get_spins(), o.get_spins())
    assert np.array_equal(g.measure(), o.measure())
    g.close()


def test_record_ring_grows_and_drains_in_order():
    case = (4, 5, 40, ig.Y_GAPBC, ig.X_FREE, 0.5, 0.0, 3.0, ig.INIT_RANDOM, 0.0)
    g, o = _pair(case)
    g.sweep(150, 1)  # more than the initial ring
    first = g.read_series(cap=40)
    g.sweep(200, 1)
    rest = g.read_series()
    want = o.sweep(350, 1)
    assert np.array_equal(np.concatenate([first, rest]), want)
    g.close()


def test_failed_ring_growth_leaves_the_film_usable():
    """A record reservation no device can hold (2^32 - 256 records of 45
    int64, about 1.5 TB) is refused with ENOMEM before anything changes: the
    pending records, the later ones (through a real ring growth) and the
    spins are still the oracle's."""
    case = (40, 6, 64, ig.Y_GAPBC, ig.X_FREE, 0.4, 0.0, 3.0, ig.INIT_SLAB_Y, 0.02)
    g, o = _pair(case)
    g.sweep(30, 1)
    with pytest.raises(ig.IsingError) as e:
        g.reserve_records(0xFFFFFF00)
    assert e.value.status == ig.ENOMEM
    g.sweep(100, 1)
    assert np.array_equal(g.read_series(), o.sweep(130, 1))
    assert np.array_equal(g.get_spins(), o.get_spins())
    g.close()


def test_failed_batch_ring_growth_leaves_the_batch_usable():
    """The same for a two-lane batch: the refused reservation (several TB)
    leaves every film's rings, records and spins as the oracle has them."""
    specs = [dict(Lx=40, Ly=4 + i, Lz=64, T=2.8 + 0.2 * i, H1=0.2, seed=23, replica=i, measure_every=1 + i,
                  init_kind=ig.INIT_SLAB_Y, flip_p=0.02) for i in range(3)]
    b = ig.Batch(specs, lanes=2)
    b.sweep(30, False)
    with pytest.raises(ig.IsingError) as e:
        b.reserve_records(0xFFFFFF00)
    assert e.value.status == ig.ENOMEM
    b.sweep(100, True)
    for i, sp in enumerate(specs):
        o = O.Film(sp["Lx"], sp["Ly"], sp["Lz"], 1.0, sp["H1"], sp["T"], sp["seed"], replica=sp["replica"])
        o.init(sp["init_kind"], sp["flip_p"])
        assert np.array_equal(b.read_series(i), o.sweep(130, sp["measure_every"])), i
        assert np.array_equal(b.get_spins(i), o.get_spins()), i
    b.close()


def test_parameter_change_between_sweeps():
    case = (6, 6, 64, ig.Y_GAPBC, ig.X_FREE, 0.5, 0.0, 3.0, ig.INIT_RANDOM, 0.0)
    g, o = _pair(case)
    g.sweep(10, 5)
    o.sweep(10, 5)
    g.set_params(1.0, 0.2, 2.2)
    o2 = O.Film(6, 6, 64, 1.0, 0.2, 2.2, 7, replica=3)
    o2.set_spins(o.get_spins())
    o2.sweep_count = o.sweep_count
    g.sweep(10, 5)
    want = o2.sweep(10, 5)
    got = g.read_series()
    assert np.array_equal(got[2:], want)
    assert np.array_equal(g.get_spins(), o2.get_spins())
    g.close()


def test_paper_scale_film_bit_exact():
    """The 120 x 240 x 1600 film (46,080,000 spins), slab start with 1% flips,
    +H1 = 0.55 at T = 3, in the launch configuration the benchmark times
    (records every 10 sweeps)."""
    Lx, Ly, Lz = 120, 240, 1600
    o = O.Film(Lx, Ly, Lz, 1.0, 0.55, 3.0, 2)
    o.init(O.INIT_SLAB_Y, 0.01)
    want = o.sweep(20, 10)
    spins = o.get_spins()
    for shape in (ig.SHAPE_GRID_1, ig.SHAPE_GRID_2, ig.SHAPE_GRID_Q):
        g = ig.Film(Lx, Ly, Lz, 1.0, 0.55, 3.0, 2, shape=shape)
        g.init(ig.INIT_SLAB_Y, 0.01)
        g.sweep(20, 10)
        assert np.array_equal(g.read_series(), want), shape
        assert np.array_equal(g.get_spins(), spins), shape
        g.close()


@pytest.mark.parametrize("shape", [ig.SHAPE_GRID_1, ig.SHAPE_GRID_2, ig.SHAPE_GRID_Q], ids=["grid1", "grid2", "gridq"])
@pytest.mark.parametrize("cold", [False, True], ids=["fast-table", "exact-table"])
def test_mixed_batch_matches_films_run_alone(cold, shape):
    """cold: one film at T -> 0 (a reachable thr = 0 entry) and one at beta = 0
    put the whole batch on the exact-table variant of the multi-film kernel."""
    specs = []
    for i, (Lx, Ly, Lz) in enumerate([(8, 8, 8), (5, 6, 66), (3, 4, 2), (7, 5, 128), (1, 8, 16), (16, 12, 96)]):
        specs.append(dict(Lx=Lx, Ly=Ly, Lz=Lz, T=2.0 + 0.3 * i, H1=0.1 * i, seed=100 + i, replica=i,
                          measure_every=(i % 3) + 1, init_kind=ig.INIT_RANDOM if i % 2 else ig.INIT_SLAB_Y,
                          flip_p=0.02, y_mode=[ig.Y_GAPBC, ig.Y_PBC, ig.Y_APBC][i % 3]))
    if cold:
        specs[1]["T"] = 1e-3
        specs[3]["T"] = math.inf
    for use_graph in (False, True):
        b = ig.Batch(specs)
        b.set_shape(shape)
        b.sweep(5, use_graph)
        b.sweep(91, use_graph)
        for i, sp in enumerate(specs):
            o = O.Film(sp["Lx"], sp["Ly"], sp["Lz"], 1.0, sp["H1"], sp["T"], sp["seed"], y_mode=sp["y_mode"],
                       replica=sp["replica"])
            o.init(sp["init_kind"], sp["flip_p"])
            want = o.sweep(96, sp["measure_every"])
            assert np.array_equal(b.read_series(i), want), (use_graph, i)
            assert np.array_equal(b.get_spins(i), o.get_spins()), (use_graph, i)
        b.close()


def test_records_when_measurement_blocks_outnumber_the_grid():
    """About 2,000 measurement blocks over 170 films -- layers grouped several
    to a block, one block per layer, two blocks per layer -- so that the
    measurement grid strides over films and the block that completes a film
    (and writes its record) is often serving another film next."""
    specs = []
    geoms = [(12, 520, 2)] * 150 + [(5, 1100, 2)] * 10 + [(6, 8, 16)] * 10
    for i, (Lx, Ly, Lz) in enumerate(geoms):
        specs.append(dict(Lx=Lx, Ly=Ly, Lz=Lz, T=2.5 + 0.01 * i, H1=0.3, seed=41, replica=i,
                          measure_every=1 + i % 3, init_kind=ig.INIT_RANDOM, y_mode=[ig.Y_GAPBC, ig.Y_PBC][i % 2]))
    b = ig.Batch(specs)
    b.set_shape(ig.SHAPE_GRID_1)
    b.sweep(12, True)
    for i, sp in enumerate(specs):
        o = O.Film(sp["Lx"], sp["Ly"], sp["Lz"], 1.0, sp["H1"], sp["T"], sp["seed"], y_mode=sp["y_mode"],
                   replica=sp["replica"])
        o.init(sp["init_kind"], 0.0)
        assert np.array_equal(b.read_series(i), o.sweep(12, sp["measure_every"])), i
    b.close()


@pytest.mark.parametrize("shape", [ig.SHAPE_GRID_1, ig.SHAPE_GRID_2, ig.SHAPE_GRID_Q], ids=["grid1", "grid2", "gridq"])
def test_records_across_call_boundaries(shape):
    """Records are summed in half-sweep 1 and written by the next half-sweep 0,
    except after a call's last sweep (a separate kernel).  Calls of one sweep
    (every record through the separate kernel), of a few sweeps and of many
    (graph chunks) alternate on one batch, with records every 1, 2 and 3
    sweeps and the seam joining one colour or not; records and spins match the
    oracle."""
    geoms = [(6, 8, 16), (7, 8, 64), (5, 6, 34), (4, 9, 96), (1, 5, 8), (9, 3, 130)]
    specs = [dict(Lx=Lx, Ly=Ly, Lz=Lz, T=2.5 + 0.2 * i, H1=0.2 * i - 0.3, seed=77, replica=i, measure_every=1 + i % 3,
                  init_kind=ig.INIT_SLAB_Y, flip_p=0.05, y_mode=[ig.Y_GAPBC, ig.Y_PBC, ig.Y_APBC][i % 3])
             for i, (Lx, Ly, Lz) in enumerate(geoms)]
    calls = [(1, False), (1, True), (3, False), (2, True), (1, False), (70, True), (1, False), (5, False)]
    b = ig.Batch(specs)
    b.set_shape(shape)
    for n, graph in calls:
        b.sweep(n, graph)
    total = sum(n for n, _ in calls)
    for i, sp in enumerate(specs):
        o = O.Film(sp["Lx"], sp["Ly"], sp["Lz"], 1.0, sp["H1"], sp["T"], sp["seed"], y_mode=sp["y_mode"],
                   replica=sp["replica"])
        o.init(sp["init_kind"], sp["flip_p"])
        want = o.sweep(total, sp["measure_every"])
        assert np.array_equal(b.read_series(i), want), i
        assert np.array_equal(b.get_spins(i), o.get_spins()), i
    b.close()


def test_thermodynamic_integration_from_gpu_records_matches_oracle():
    """The film's own integral over H1 (8 Gauss-Legendre nodes): the FP64 result from the GPU's
    records through the library equals the oracle-fed numpy result to 1e-12."""
    from oracle import ti as OT
    H1max, n = 0.6, 8
    xs, _ = ig.gauss_legendre(n, 0.0, H1max)
    specs = [dict(Lx=6, Ly=8, Lz=16, T=3.0, H1=float(h), seed=5, replica=r, measure_every=1, y_mode=ig.Y_PBC,
                  init_kind=ig.INIT_ALL_UP) for r, h in enumerate(xs)]
    b = ig.Batch(specs)
    b.sweep(300, True)
    m1g, mng, m1o, mno = [], [], [], []
    area = 8 * 16
    for i, sp in enumerate(specs):
        r = b.read_series(i)
        o = O.Film(6, 8, 16, 1.0, sp["H1"], 3.0, 5, y_mode=O.Y_PBC, replica=i)
        o.init(O.INIT_ALL_UP)
        ro = o.sweep(300, 1)
        assert np.array_equal(r, ro)
        m1g.append(ig.series_mean(r, 3, first=50) / area)
        mng.append(ig.series_mean(r, 4, first=50) / area)
        m1o.append(OT.series_mean(ro, 3, first=50) / area)
        mno.append(OT.series_mean(ro, 4, first=50) / area)
    a = ig.ti_surface_field(H1max, m1g, mng)
    c = OT.surface_field_ti(H1max, m1o, mno)
    assert abs(a - c) <= 1e-12 * abs(c)
    b.close()


def test_shape_limits_and_switches():
    """The resident kernel is refused for a film it cannot hold; a film can
    change launch shape (the cluster kernel included) in the middle of its
    chain."""
    big = ig.Film(64, 64, 32, 1.0, 0.5, 3.0, 1)  # 131072 spins
    with pytest.raises(ig.IsingError) as e:
        big.set_shape(ig.SHAPE_RESIDENT)
    assert e.value.status == ig.EINVAL
    assert big.get_shape(1) in (ig.SHAPE_GRID_1, ig.SHAPE_GRID_2)
    big.close()
    case = (12, 10, 40, ig.Y_GAPBC, ig.X_FREE, 0.55, 0.0, 3.0, ig.INIT_SLAB_Y, 0.01)
    g, o = _pair(case)
    for shape, n, m in ((ig.SHAPE_RESIDENT, 7, 2), (ig.SHAPE_GRID_2, 5, 3), (ig.SHAPE_GRID_1, 4, 4),
                        (ig.SHAPE_CLUSTER, 9, 2), (ig.SHAPE_GRID_Q, 6, 2), (ig.SHAPE_CLUSTER, 3, 1),
                        (ig.SHAPE_RESIDENT, 11, 1)):
        g.set_shape(shape)
        g.sweep(n, m)
        assert np.array_equal(g.read_series(), o.sweep(n, m))
        assert np.array_equal(g.get_spins(), o.get_spins())
    g.close()


def test_autotune_leaves_the_chain_alone():
    """ising_autotune runs on a scratch film: the tuned film's chain is still
    the oracle's, the choice is a valid shape, and another AUTO film of the
    same shape and record interval picks it up from the process table."""
    case = (20, 24, 40, ig.Y_GAPBC, ig.X_FREE, 0.45, 0.0, 3.0, ig.INIT_SLAB_Y, 0.01)
    g, o = _pair(case)
    g.sweep(3, 1)
    want = [o.sweep(3, 1)]
    best = g.autotune(1)
    assert best in SHAPES
    g.sweep(9, 1)
    want.append(o.sweep(9, 1))
    assert np.array_equal(g.read_series(), np.concatenate(want))
    assert np.array_equal(g.get_spins(), o.get_spins())
    g.close()
    g, o = _pair(case)
    assert g.get_shape(1) == best
    g.sweep(12, 1)
    assert np.array_equal(g.read_series(), o.sweep(12, 1))
    assert np.array_equal(g.get_spins(), o.get_spins())
    g.close()


def test_batch_autotune_leaves_the_chains_alone():
    specs = [dict(Lx=Lx, Ly=Ly, Lz=Lz, T=3.0, H1=0.3, seed=9, replica=i, measure_every=2,
                  init_kind=ig.INIT_SLAB_Y, flip_p=0.02) for i, (Lx, Ly, Lz) in enumerate([(8, 16, 32), (12, 20, 64)])]
    b = ig.Batch(specs)
    b.sweep(4, True)
    best = b.autotune()
    assert best in (ig.SHAPE_GRID_1, ig.SHAPE_GRID_2, ig.SHAPE_GRID_Q, ig.SHAPE_CLUSTER) and b.get_shape() == best
    b.sweep(40, True)
    for i, sp in enumerate(specs):
        o = O.Film(sp["Lx"], sp["Ly"], sp["Lz"], 1.0, sp["H1"], sp["T"], sp["seed"], replica=sp["replica"])
        o.init(sp["init_kind"], sp["flip_p"])
        assert np.array_equal(b.read_series(i), o.sweep(44, 2))
        assert np.array_equal(b.get_spins(i), o.get_spins())
    b.close()


def test_async_record_reads_match_the_oracle():
    """ising_read_series_async: one record per step copied to pinned host
    memory while later steps run (through several wraps of the 64-record
    ring), then a ring growth with a copy still in flight, then synchronous
    reads; every record equals the oracle's."""
    torch = pytest.importorskip("torch")
    case = (6, 8, 40, ig.Y_GAPBC, ig.X_FREE, 0.5, 0.0, 3.0, ig.INIT_SLAB_Y, 0.01)
    for shape in (ig.SHAPE_RESIDENT, ig.SHAPE_GRID_1):
        g, o = _pair(case, shape=shape)
        rl = 5 + case[0]
        host = torch.zeros((300, rl), dtype=torch.int64).pin_memory()
        n = 0
        for i in range(150):
            g.sweep(2, 2)
            n += g.read_series_async(host[n].data_ptr(), 1)
        assert n == 150
        g.sweep(20, 1)
        k = g.read_series_async(host[150].data_ptr(), 10)  # in flight while the ring grows below
        g.sweep(300, 1)
        rest = g.read_series()
        g.synchronize()
        want = o.sweep(300, 2)
        assert np.array_equal(host[:150].numpy(), want)
        want = np.concatenate([o.sweep(20, 1), o.sweep(300, 1)])
        assert k == 10 and np.array_equal(host[150:160].numpy(), want[:10])
        assert np.array_equal(rest, want[10:])
        assert np.array_equal(g.get_spins(), o.get_spins())
        g.close()


@pytest.mark.parametrize("lanes", [1, 2, 3, 5])
def test_lanes_give_the_same_chains(lanes):
    """However the films are spread over lanes, every film's records and spins
    are the oracle's (direct and graph calls, records every 1-3 sweeps, a
    shape pinned and the autotuner's)."""
    geoms = [(6, 8, 16), (12, 20, 64), (5, 6, 34), (4, 9, 96), (1, 5, 8), (9, 3, 130), (16, 12, 96)]
    specs = [dict(Lx=Lx, Ly=Ly, Lz=Lz, T=2.2 + 0.3 * i, H1=0.1 * i, seed=31, replica=i, measure_every=1 + i % 3,
                  init_kind=ig.INIT_RANDOM if i % 2 else ig.INIT_SLAB_Y, flip_p=0.02,
                  y_mode=[ig.Y_GAPBC, ig.Y_PBC, ig.Y_APBC][i % 3]) for i, (Lx, Ly, Lz) in enumerate(geoms)]
    b = ig.Batch(specs, lanes=lanes)
    assert b.lanes == min(lanes, len(specs))
    b.set_shape(ig.SHAPE_GRID_2)
    b.sweep(7, False)
    b.autotune()
    b.sweep(100, True)
    for i, sp in enumerate(specs):
        o = O.Film(sp["Lx"], sp["Ly"], sp["Lz"], 1.0, sp["H1"], sp["T"], sp["seed"], y_mode=sp["y_mode"],
                   replica=sp["replica"])
        o.init(sp["init_kind"], sp["flip_p"])
        want = o.sweep(107, sp["measure_every"])
        assert np.array_equal(b.read_series(i), want), i
        assert np.array_equal(b.get_spins(i), o.get_spins()), i
    b.close()


def test_batch_rings_grow_with_wrapped_unread_records():
    """Two lanes; records every 1, 2, 1 and 3 sweeps; partial reads leave
    unread records that wrap round a ring, and a later call grows that ring
    (graph and direct calls).  Every film's full series, read in pieces, and
    its final spins equal the oracle's."""
    geoms = [(6, 8, 40), (5, 6, 34), (8, 10, 64), (4, 9, 96)]
    every = [1, 2, 1, 3]
    specs = [dict(Lx=Lx, Ly=Ly, Lz=Lz, T=2.6 + 0.2 * i, H1=0.15 * i, seed=17, replica=i, measure_every=m,
                  init_kind=ig.INIT_SLAB_Y, flip_p=0.02) for i, ((Lx, Ly, Lz), m) in enumerate(zip(geoms, every))]
    b = ig.Batch(specs, lanes=2)
    got = [[] for _ in specs]

    def read(i, cap=None):
        r = b.read_series(i) if cap is None else b.read_series(i, cap=cap)
        got[i].append(r)
        return len(r)

    b.sweep(100, True)  # rings of the every-sweep films grow from 64 records
    assert read(0, cap=30) == 30
    read(1)
    read(3, cap=5)
    b.sweep(20, False)
    b.sweep(30, False)  # film 0's unread records now wrap round its ring
    assert read(0, cap=50) == 50
    b.sweep(150, True)  # ...and that ring grows with them in it
    for i in range(len(specs)):
        read(i)
    for i, sp in enumerate(specs):
        o = O.Film(sp["Lx"], sp["Ly"], sp["Lz"], 1.0, sp["H1"], sp["T"], sp["seed"], replica=sp["replica"])
        o.init(sp["init_kind"], sp["flip_p"])
        want = o.sweep(300, sp["measure_every"])
        assert np.array_equal(np.concatenate(got[i]), want), i
        assert np.array_equal(b.get_spins(i), o.get_spins()), i
    b.close()


def test_lanes_join_the_batch_stream():
    """Work queued on the batch's stream after a sweep sees every lane's
    films swept: a torch copy of a lane-1 film's spins taken on that stream
    right after the sweep call matches the final lattice."""
    torch = pytest.importorskip("torch")
    specs = [dict(Lx=8, Ly=10, Lz=64, T=3.0, H1=0.2, seed=5, replica=i, measure_every=0) for i in range(4)]
    st = torch.cuda.Stream()
    b = ig.Batch(specs, stream=st, lanes=2)
    b.sweep(40, True)
    done = torch.cuda.Event()
    done.record(st)
    done.synchronize()
    for i, sp in enumerate(specs):
        o = O.Film(8, 10, 64, 1.0, 0.2, 3.0, 5, replica=i)
        o.init(O.INIT_RANDOM)
        o.sweep(40, 0)
        assert np.array_equal(b.get_spins(i), o.get_spins()), i
    b.close()
