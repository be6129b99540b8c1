"""ising_measure_packed_noalloc: the allocation-free record of a packed film.

Callers that cannot allocate device memory (their pool allocator owns the
device, or they cannot take cudaMalloc's implicit synchronisation) get the
same record as ising_measure from a library-owned fixed scratch array.  The
check, for every y rule, periodic x, Lz = 2, a film whose layers need
several measurement blocks and a film at exactly the 8192 blocks the array
holds: two calls in a row, on states a few sweeps apart, each equal to the
oracle's record of the same spins and to ising_measure.  Collected last so
that a failing run has already exercised every other test.
"""
import ctypes

import numpy as np
import pytest

import paper_1411_5588_gb300 as ig
from oracle import oracle as O

pytestmark = pytest.mark.gpu

# (Lx, Ly, Lz, y_mode, x_mode): measurement blocks = Lx * ceil(Ly * ceil(Lz / 64) / 1024)
FILMS = [
    (24, 32, 130, ig.Y_GAPBC, ig.X_FREE),
    (24, 32, 130, ig.Y_PBC, ig.X_FREE),
    (23, 30, 130, ig.Y_APBC, ig.X_FREE),
    (12, 18, 70, ig.Y_GAPBC, ig.X_PBC),
    (7, 9, 2, ig.Y_GAPBC, ig.X_FREE),
    (8, 256, 512, ig.Y_GAPBC, ig.X_FREE),   # Ly * W = 2048: two blocks per layer
    (8192, 4, 2, ig.Y_GAPBC, ig.X_FREE),    # 8192 blocks: the whole scratch array
]


def _noalloc_record(film, torch, y_mode, x_mode, sweep):
    packed = torch.empty(film.packed_words(), dtype=torch.int32, device="cuda")
    rec = torch.zeros(5 + film.Lx, dtype=torch.int64, device="cuda")
    film.get_packed_device(packed.data_ptr())
    film.synchronize()
    P = ctypes.c_void_p
    ig.check(ig.lib().ising_measure_packed_noalloc(P(packed.data_ptr()), film.Lx, film.Ly, film.Lz, y_mode, x_mode,
                                                   sweep, P(rec.data_ptr()), None),
             "ising_measure_packed_noalloc")
    torch.cuda.synchronize()
    return rec.cpu().numpy()


def _oracle_record(film, y_mode, x_mode, spins, sweep):
    o = O.Film(film.Lx, film.Ly, film.Lz, 1.0, 0.45, 2.8, 13, y_mode=y_mode, x_mode=x_mode)
    o.set_spins(spins)
    o.sweep_count = sweep
    return o.measure()


@pytest.mark.parametrize("Lx,Ly,Lz,y_mode,x_mode", FILMS)
def test_noalloc_record_matches_the_oracle_twice(Lx, Ly, Lz, y_mode, x_mode):
    torch = pytest.importorskip("torch")
    torch.cuda.init()
    film = ig.Film(Lx, Ly, Lz, 1.0, 0.45, 2.8, 13, y_mode=y_mode, x_mode=x_mode)
    film.init(ig.INIT_SLAB_Y, 0.05)
    for n in (5, 7):
        film.sweep(n, 0)
        got = _noalloc_record(film, torch, y_mode, x_mode, film.sweep_count)
        want = _oracle_record(film, y_mode, x_mode, film.get_spins(), film.sweep_count)
        assert np.array_equal(got, want), (got[:5], want[:5])
        assert np.array_equal(got, film.measure())
    film.close()


def test_noalloc_rejects_films_beyond_the_fixed_scratch():
    # 8193 layers need 8193 measurement blocks, one more than the array holds
    rc = ig.lib().ising_measure_packed_noalloc(ctypes.c_void_p(16), 8193, 4, 2, ig.Y_GAPBC, ig.X_FREE, 0,
                                               ctypes.c_void_p(16), None)
    assert rc == ig.EINVAL
    assert b"scratch" in ig.lib().ising_last_error()
