"""ising_measure_packed_noalloc: the allocation-free record of a packed film.

Callers that cannot allocate device memory (their pool allocator owns the
device, or they cannot take cudaMalloc's implicit synchronisation) get the
same record as ising_measure from a library-owned fixed scratch array.  The
check: two calls in a row, on states two sweep batches apart, each equal to
ising_measure of the same film.  Collected last so that a failing run has
already exercised every other test.
"""
import ctypes

import numpy as np
import pytest

import paper_1411_5588_gb300 as ig

pytestmark = pytest.mark.gpu


def _noalloc_record(film, torch, sweep):
    words = film.packed_words()
    packed = torch.empty(words, dtype=torch.int32, device="cuda")
    rec = torch.zeros(5 + film.Lx, dtype=torch.int64, device="cuda")
    film.get_packed_device(packed.data_ptr())
    film.synchronize()
    P = ctypes.c_void_p
    ig.check(ig.lib().ising_measure_packed_noalloc(P(packed.data_ptr()), film.Lx, film.Ly, film.Lz, ig.Y_GAPBC,
                                                   ig.X_FREE, sweep, P(rec.data_ptr()), None),
             "ising_measure_packed_noalloc")
    torch.cuda.synchronize()
    return rec.cpu().numpy()


def test_noalloc_record_matches_ising_measure_twice():
    torch = pytest.importorskip("torch")
    torch.cuda.init()
    film = ig.Film(24, 32, 130, 1.0, 0.45, 2.8, 13, y_mode=ig.Y_GAPBC)
    film.init(ig.INIT_SLAB_Y, 0.05)
    for n in (5, 7):
        film.sweep(n, 0)
        want = film.measure()
        got = _noalloc_record(film, torch, film.sweep_count)
        assert np.array_equal(got, want), (got, want)
    film.close()


def test_noalloc_rejects_films_beyond_the_fixed_scratch():
    # 9000 layers need 9000 measurement blocks, more than the 8192 the array holds
    rc = ig.lib().ising_measure_packed_noalloc(ctypes.c_void_p(16), 9000, 4, 4, ig.Y_GAPBC, ig.X_FREE, 0,
                                               ctypes.c_void_p(16), None)
    assert rc == ig.EINVAL
    assert b"scratch" in ig.lib().ising_last_error()
