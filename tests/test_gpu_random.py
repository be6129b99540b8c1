"""Randomised parity: films with random geometry (ragged last words, tiny
sizes, both parities of Lx + Ly), boundary modes, fields, temperatures
(including T -> 0 and beta = 0), initial states, launch shapes and record
intervals, run in several calls, each bit-identical to the oracle; and the
same films as one batch, on a random grid shape."""
import math

import numpy as np
import pytest

import paper_1411_5588_gb300 as ig
from oracle import oracle as O

pytestmark = pytest.mark.gpu

SHAPES = [ig.SHAPE_AUTO, ig.SHAPE_RESIDENT, ig.SHAPE_GRID_1, ig.SHAPE_GRID_2, ig.SHAPE_GRID_Q, ig.SHAPE_CLUSTER]


def _films(seed, n):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        Lx = int(rng.integers(1, 13))
        Ly = int(rng.integers(2, 14))
        Lz = 2 * int(rng.integers(1, 90))
        x_mode = ig.X_PBC if (Lx % 2 == 0 and rng.random() < 0.2) else ig.X_FREE
        T = float(rng.choice([1e-3, math.inf, rng.uniform(1.0, 6.0), rng.uniform(1.0, 6.0)]))
        out.append(dict(Lx=Lx, Ly=Ly, Lz=Lz, y_mode=int(rng.integers(0, 3)), x_mode=x_mode,
                        H1=float(rng.uniform(-1.0, 1.0)), H=float(rng.choice([0.0, rng.uniform(-0.3, 0.3)])),
                        T=T, seed=int(rng.integers(1, 1 << 40)), replica=i,
                        init_kind=int(rng.integers(0, 3)), flip_p=float(rng.choice([0.0, 0.01, 0.5])),
                        shape=SHAPES[int(rng.integers(0, len(SHAPES)))],
                        calls=[(int(rng.integers(1, 30)), int(rng.integers(0, 5))) for _ in range(3)]))
    return out


def _oracle(f):
    o = O.Film(f["Lx"], f["Ly"], f["Lz"], 1.0, f["H1"], f["T"], f["seed"], y_mode=f["y_mode"],
               x_mode=f["x_mode"], H=f["H"], replica=f["replica"])
    o.init(f["init_kind"], f["flip_p"])
    return o


@pytest.mark.parametrize("seed", [11, 12, 14, 15, 16, 17])
def test_random_single_films(seed):
    for f in _films(seed, 20):
        g = ig.Film(f["Lx"], f["Ly"], f["Lz"], 1.0, f["H1"], f["T"], f["seed"], y_mode=f["y_mode"],
                    x_mode=f["x_mode"], H=f["H"], replica=f["replica"])
        if f["shape"] == ig.SHAPE_RESIDENT and f["Lx"] * f["Ly"] * f["Lz"] > 65536:
            f["shape"] = ig.SHAPE_GRID_1
        g.set_shape(f["shape"])
        o = _oracle(f)
        g.init(f["init_kind"], f["flip_p"])
        for n, m in f["calls"]:
            g.sweep(n, m)
            want = o.sweep(n, m)
            got = g.read_series()
            assert np.array_equal(got, want), f
        assert np.array_equal(g.get_spins(), o.get_spins()), f
        g.close()


@pytest.mark.parametrize("seed", [13, 18])
def test_random_batch(seed):
    films = _films(seed, 24)
    n = 37
    specs = [dict(f, measure_every=(i % 4)) for i, f in enumerate(films)]
    b = ig.Batch(specs)
    b.set_shape([ig.SHAPE_GRID_1, ig.SHAPE_GRID_2, ig.SHAPE_GRID_Q][len(specs) % 3])
    b.sweep(n, True)
    for i, sp in enumerate(specs):
        o = _oracle(sp)
        want = o.sweep(n, sp["measure_every"])
        assert np.array_equal(b.read_series(i), want), sp
        assert np.array_equal(b.get_spins(i), o.get_spins()), sp
    b.close()


@pytest.mark.parametrize("seed", [21, 22, 23])
def test_random_batch_chains(seed):
    """Random films in a random number of lanes, driven by a random sequence
    of calls: short and long sweeps, direct and graph, records every 0-4
    sweeps, the launch shape switched between calls, records read part-way.
    Every film's records and final spins are the oracle's."""
    rng = np.random.default_rng(seed)
    films = _films(seed, 16)
    specs = [dict(f, measure_every=int(rng.integers(0, 5))) for f in films]
    lanes = int(rng.integers(1, 5))
    b = ig.Batch(specs, lanes=lanes)
    assert b.lanes == min(lanes, len(specs))
    shapes = [ig.SHAPE_GRID_1, ig.SHAPE_GRID_2, ig.SHAPE_GRID_Q]
    oracles = [_oracle(sp) for sp in specs]
    got = [[] for _ in specs]
    want = [[] for _ in specs]
    for _ in range(6):
        b.set_shape(shapes[int(rng.integers(0, 3))])
        n = int(rng.choice([1, 2, 5, 33, 70]))
        b.sweep(n, bool(rng.integers(0, 2)))
        for i, sp in enumerate(specs):
            want[i].append(oracles[i].sweep(n, sp["measure_every"]))
        if rng.random() < 0.5:  # read everything pending so far
            for i in range(len(specs)):
                got[i].append(b.read_series(i))
    for i, sp in enumerate(specs):
        got[i].append(b.read_series(i))
        g = np.concatenate(got[i]) if got[i] else np.zeros((0, 5 + sp["Lx"]), dtype=np.int64)
        w = np.concatenate(want[i])
        assert np.array_equal(g, w), (seed, i, sp)
        assert np.array_equal(b.get_spins(i), oracles[i].get_spins()), (seed, i, sp)
    b.close()
