"""The cluster-resident path (ISING_SHAPE_CLUSTER) against the CPU oracle, bit
for bit.

A thread-block cluster of C CTAs keeps a film of a batch in distributed
shared memory for a whole call, CTA r holding a slab of layers, then takes
its next film; a word's
x-neighbour across a slab boundary, and the mirrored layer of an Eq. 11
partner row, come from a peer CTA.  So the cases cover every cluster size
with slabs of one layer and of several, uneven slabs (Lx not a multiple of
C), the Eq. 11 wrap joining equal and opposite colours (both parities of
Lx + Ly), periodic and antiperiodic y, periodic x (its wrap across the first
and last slab), ragged last words, Lz = 2, Ly = 2, Lx = 1 and the degenerate
temperatures beta = 0 and T -> 0 (the exact-table variant); records every
1-3 sweeps across call boundaries (a record's sums are reduced over the
cluster in the half-sweep after the one that took them, or after the call's
last sweep); and switches between the grid kernels and the cluster path in
mid-chain.
"""
import math

import numpy as np
import pytest

import paper_1411_5588_gb300 as ig
from oracle import oracle as O

pytestmark = pytest.mark.gpu

#        Lx  Ly  Lz   y_mode      x_mode    H1     H     T      init            flip
FILMS = [
    (8, 8, 8, ig.Y_GAPBC, ig.X_FREE, 0.5, 0.0, 3.0, ig.INIT_RANDOM, 0.0),
    (9, 6, 66, ig.Y_GAPBC, ig.X_FREE, 0.55, 0.0, 2.5, ig.INIT_RANDOM, 0.0),
    (8, 4, 2, ig.Y_GAPBC, ig.X_FREE, 0.3, 0.0, 2.0, ig.INIT_RANDOM, 0.0),
    (10, 3, 130, ig.Y_PBC, ig.X_FREE, 0.2, 0.0, 3.5, ig.INIT_RANDOM, 0.0),
    (8, 2, 64, ig.Y_APBC, ig.X_FREE, 0.4, 0.0, 3.0, ig.INIT_RANDOM, 0.0),
    (11, 5, 128, ig.Y_GAPBC, ig.X_FREE, 0.45, 0.0, 3.0, ig.INIT_SLAB_Y, 0.01),
    (8, 4, 8, ig.Y_PBC, ig.X_PBC, 0.0, 0.0, 4.5, ig.INIT_RANDOM, 0.0),
    (9, 10, 190, ig.Y_GAPBC, ig.X_FREE, -0.3, 0.1, 1.5, ig.INIT_SLAB_Y, 0.01),
    (12, 9, 34, ig.Y_APBC, ig.X_PBC, 0.25, -0.2, 2.8, ig.INIT_RANDOM, 0.0),
    (16, 12, 96, ig.Y_GAPBC, ig.X_FREE, 0.55, 0.0, 3.0, ig.INIT_SLAB_Y, 0.01),
    (13, 16, 12, ig.Y_GAPBC, ig.X_FREE, -0.5, 0.0, 2.3, ig.INIT_SLAB_Y, 0.01),
    (32, 24, 64, ig.Y_GAPBC, ig.X_FREE, 0.55, 0.0, 3.0, ig.INIT_SLAB_Y, 0.0),
]


def _spec(f, i, measure_every, T=None):
    Lx, Ly, Lz, y_mode, x_mode, H1, H, T0, init, flip = f
    return dict(Lx=Lx, Ly=Ly, Lz=Lz, y_mode=y_mode, x_mode=x_mode, H1=H1, H=H, T=T0 if T is None else T,
                seed=500 + i, replica=i, init_kind=init, flip_p=flip, measure_every=measure_every)


def _oracle(sp):
    o = O.Film(sp["Lx"], sp["Ly"], sp["Lz"], 1.0, sp["H1"], sp["T"], sp["seed"], y_mode=sp["y_mode"],
               x_mode=sp.get("x_mode", ig.X_FREE), H=sp.get("H", 0.0), replica=sp["replica"])
    o.init(sp["init_kind"], sp["flip_p"])
    return o


def _check(b, specs, calls):
    total = sum(n for n, _ in calls)
    for i, sp in enumerate(specs):
        o = _oracle(sp)
        want = o.sweep(total, sp["measure_every"])
        assert np.array_equal(b.read_series(i), want), (i, sp)
        assert np.array_equal(b.get_spins(i), o.get_spins()), (i, sp)


@pytest.mark.parametrize("C", [1, 2, 3, 4, 8])
@pytest.mark.parametrize("cold", [False, True], ids=["fast-table", "exact-table"])
def test_cluster_batch_bit_exact(C, cold):
    """Every film with at least C layers, C CTAs each, records every 1-3
    sweeps, over calls of 1, 4 and 37 sweeps; cold: one film at T -> 0 and
    one at beta = 0 put the launch on the exact-table variant."""
    films = [f for f in FILMS if f[0] >= C]
    specs = [_spec(f, i, 1 + i % 3) for i, f in enumerate(films)]
    if cold:
        specs[0]["T"] = 1e-3
        specs[-1]["T"] = math.inf
    calls = [(1, False), (4, True), (37, False)]
    b = ig.Batch(specs, lanes=1)
    b.set_cluster_size(C)
    b.set_shape(ig.SHAPE_CLUSTER)
    assert b.get_shape() == ig.SHAPE_CLUSTER and b.cluster_size == C
    for n, g in calls:
        b.sweep(n, g)
    _check(b, specs, calls)
    b.close()


def test_cluster_odd_sizes_and_one_layer_slabs():
    """Lx = C (one layer per CTA, every x-neighbour remote), Lx = 1 on one
    CTA, and slabs of uneven length (Lx = 7 over 3 and 5 CTAs)."""
    cases = [((5, 6, 20, ig.Y_GAPBC, ig.X_FREE, 0.4, 0.0, 2.7, ig.INIT_RANDOM, 0.0), 5),
             ((4, 7, 64, ig.Y_GAPBC, ig.X_PBC, 0.3, 0.0, 3.1, ig.INIT_RANDOM, 0.0), 4),
             ((1, 8, 16, ig.Y_GAPBC, ig.X_FREE, 0.7, 0.0, 2.2, ig.INIT_RANDOM, 0.0), 1),
             ((7, 5, 98, ig.Y_GAPBC, ig.X_FREE, 0.6, 0.0, 2.4, ig.INIT_SLAB_Y, 0.02), 3),
             ((7, 6, 98, ig.Y_GAPBC, ig.X_FREE, 0.6, 0.0, 2.4, ig.INIT_SLAB_Y, 0.02), 5),
             ((6, 2, 2, ig.Y_APBC, ig.X_FREE, 0.1, 0.0, 3.0, ig.INIT_RANDOM, 0.0), 6)]
    for k, (f, C) in enumerate(cases):
        specs = [_spec(f, k, 1 + k % 2)]
        b = ig.Batch(specs, lanes=1)
        b.set_cluster_size(C)
        b.set_shape(ig.SHAPE_CLUSTER)
        calls = [(3, False), (20, False)]
        for n, g in calls:
            b.sweep(n, g)
        _check(b, specs, calls)
        b.close()


@pytest.mark.parametrize("seed", [31, 32])
def test_cluster_and_grid_shapes_alternate(seed):
    """The same batch switched between the grid kernels and the cluster path
    (automatic and pinned cluster sizes) between calls, in one to three lanes,
    with records read part-way: every film's records and spins are the
    oracle's."""
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(12):
        Lx = int(rng.integers(4, 20))
        Ly = int(rng.integers(2, 14))
        Lz = 2 * int(rng.integers(1, 90))
        x_mode = ig.X_PBC if (Lx % 2 == 0 and rng.random() < 0.2) else ig.X_FREE
        T = float(rng.choice([1e-3, math.inf, rng.uniform(1.0, 6.0), rng.uniform(1.0, 6.0)]))
        specs.append(dict(Lx=Lx, Ly=Ly, Lz=Lz, y_mode=int(rng.integers(0, 3)), x_mode=x_mode,
                          H1=float(rng.uniform(-1.0, 1.0)), H=float(rng.choice([0.0, rng.uniform(-0.3, 0.3)])), T=T,
                          seed=int(rng.integers(1, 1 << 40)), replica=i, init_kind=int(rng.integers(0, 3)),
                          flip_p=float(rng.choice([0.0, 0.01, 0.5])), measure_every=int(rng.integers(0, 4))))
    b = ig.Batch(specs, lanes=int(rng.integers(1, 4)))
    oracles = [_oracle(sp) for sp in specs]
    got = [[] for _ in specs]
    want = [[] for _ in specs]
    for step in range(6):
        choice = int(rng.integers(0, 4))
        if choice == 0:
            b.set_shape(ig.SHAPE_GRID_1)
        elif choice == 1:
            b.set_shape(ig.SHAPE_GRID_2)
        else:
            b.set_cluster_size(int(rng.integers(1, 5)) if choice == 3 else 0)
            b.set_shape(ig.SHAPE_CLUSTER)
        n = int(rng.choice([1, 2, 5, 33]))
        b.sweep(n, bool(rng.integers(0, 2)))
        for i, sp in enumerate(specs):
            want[i].append(oracles[i].sweep(n, sp["measure_every"]))
        if rng.random() < 0.5:
            for i in range(len(specs)):
                got[i].append(b.read_series(i))
    for i, sp in enumerate(specs):
        got[i].append(b.read_series(i))
        g = np.concatenate(got[i])
        w = np.concatenate(want[i])
        assert np.array_equal(g, w), (seed, i, sp)
        assert np.array_equal(b.get_spins(i), oracles[i].get_spins()), (seed, i, sp)
    b.close()


@pytest.mark.parametrize("C", [1, 4, 8])
def test_clusters_take_several_films_in_turn(C):
    """Sixteen lanes: each lane gets n_SM / (C x 16) clusters (one for C = 8
    on 152 SMs), fewer than its films, so a cluster sweeps two or more films
    one after another, every sweep of the call for each, records included;
    films of every size share a cluster (largest-first packing)."""
    films = [f for f in FILMS if f[0] >= C]
    specs = [_spec(films[i % len(films)], i, 1 + i % 3) for i in range(40)]
    b = ig.Batch(specs, lanes=16)
    b.set_cluster_size(C)
    b.set_shape(ig.SHAPE_CLUSTER)
    calls = [(2, False), (9, True)]
    for n, g in calls:
        b.sweep(n, g)
    _check(b, specs, calls)
    b.close()


def test_contact_angle_films_on_clusters():
    """Films of the contact-angle set's geometry (32 x 96 x 64: one word per
    row array, the Eq. 11 film from a slab start and periodic-y films from
    all up) on clusters of 3 CTAs, a record after every sweep."""
    from paper_1411_5588_gb300 import workloads as WL
    s = WL.contact_angle_set(H1s=(0.3,), n_gl=2, n_sweeps=30)
    specs = s["jobs"]
    b = ig.Batch(specs, lanes=1)
    b.set_cluster_size(3)
    b.set_shape(ig.SHAPE_CLUSTER)
    b.sweep(30, False)
    _check(b, specs, [(30, False)])
    b.close()


def test_cluster_size_limits():
    specs = [_spec(FILMS[0], 0, 1), _spec(FILMS[1], 1, 0)]
    b = ig.Batch(specs, lanes=1)
    with pytest.raises(ig.IsingError) as e:
        b.set_cluster_size(9)
    assert e.value.status == ig.EINVAL
    b.set_cluster_size(8)  # Lx = 8 and 9: both qualify
    b.set_shape(ig.SHAPE_CLUSTER)
    assert b.cluster_size == 8
    b.set_shape(ig.SHAPE_GRID_1)
    assert b.cluster_size == 0 and b.get_shape() == ig.SHAPE_GRID_1
    b.close()
    thin = [_spec((3, 4, 2, ig.Y_GAPBC, ig.X_FREE, 0.3, 0.0, 2.0, ig.INIT_RANDOM, 0.0), 0, 1)]
    b = ig.Batch(thin, lanes=1)
    with pytest.raises(ig.IsingError) as e:
        b.set_cluster_size(4)  # three layers cannot fill four CTAs
    assert e.value.status == ig.EINVAL
    b.set_shape(ig.SHAPE_CLUSTER)  # automatic: three CTAs at most
    assert 1 <= b.cluster_size <= 3
    b.sweep(9, False)
    _check(b, thin, [(9, False)])
    b.close()


@pytest.mark.parametrize("small", [False, True], ids=["mixed-films", "two-small-films"])
def test_autotune_with_cluster_candidates_leaves_the_chains_alone(small):
    """The autotuner may pick the cluster path (two small films, where a
    grid half-sweep is mostly launch overhead, usually take it); a size
    pinned afterwards applies at once, and 0 restores the autotuner's."""
    films = FILMS[:2] if small else FILMS
    specs = [_spec(f, i, 1) for i, f in enumerate(films)]
    b = ig.Batch(specs)
    shape = b.autotune()
    assert shape in (ig.SHAPE_GRID_1, ig.SHAPE_GRID_2, ig.SHAPE_GRID_Q, ig.SHAPE_CLUSTER)
    assert b.get_shape() == shape
    calls = [(17, True)]
    b.sweep(17, True)
    if shape == ig.SHAPE_CLUSTER:
        tuned = b.cluster_size
        b.set_cluster_size(1)
        assert b.cluster_size == 1
        b.sweep(5, False)
        b.set_cluster_size(0)
        assert b.cluster_size == tuned
        calls.append((5, False))
    _check(b, specs, calls)
    b.close()


def test_cluster_slab_at_the_shared_memory_limit():
    """A film whose slab on 8 CTAs needs exactly the 200 KiB a CTA may take
    (64 x 1588 x 128: 8 layers x 1588 rows x 2 words x 2 planes x 4 B, plus
    24 B per layer of tables) runs bit-exact; one row more is refused for 8
    CTAs, and then for every size (fewer CTAs hold larger slabs): EINVAL,
    and the batch stays on the grid kernels."""
    sp = dict(Lx=64, Ly=1588, Lz=128, y_mode=ig.Y_GAPBC, x_mode=ig.X_FREE, H1=0.5, H=0.0, T=3.0, seed=11,
              replica=0, init_kind=ig.INIT_SLAB_Y, flip_p=0.01, measure_every=1)
    b = ig.Batch([sp], lanes=1)
    b.set_cluster_size(8)
    b.set_shape(ig.SHAPE_CLUSTER)
    assert b.cluster_size == 8
    b.sweep(3, False)
    _check(b, [sp], [(3, False)])
    b.close()
    big = dict(sp, Ly=1589)
    b = ig.Batch([big], lanes=1)
    with pytest.raises(ig.IsingError) as e:
        b.set_cluster_size(8)
    assert e.value.status == ig.EINVAL
    with pytest.raises(ig.IsingError) as e:
        b.set_shape(ig.SHAPE_CLUSTER)
    assert e.value.status == ig.EINVAL
    assert b.cluster_size == 0 and b.get_shape() == ig.SHAPE_GRID_1
    b.close()
