"""GPU path vs the oracle on the benchmark workloads at their full sizes.

  - the 8^3 film over its whole run (10^4 sweeps, a record every sweep);
  - the 64-film integration set in one batch, in the launch shape the
    benchmark's autotuner picks for it: full spin/record parity for two films
    of each size, and for every other film its last record equals the
    oracle's measurement of its final spins;
  - the hottest and coldest films of the 40-film temperature scan (full
    parity), and for every fourth film the same last-record check;
  - the first jobs of the 2000-job stream through the server (their sweep
    counts cut to a few so that the oracle can follow).
"""
import numpy as np
import pytest

import paper_1411_5588_gb300 as ig
from oracle import oracle as O
from paper_1411_5588_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


def _oracle(job, n, m):
    o = O.Film(job["Lx"], job["Ly"], job["Lz"], job["J"], job["H1"], job["T"], job["seed"],
               y_mode=job["y_mode"], replica=job["replica"])
    o.init(job["init_kind"], job["flip_p"])
    return o, o.sweep(n, m)


def _measured(job, spins, sweep):
    """The oracle's record of a given lattice (stamped with `sweep`)."""
    o = O.Film(job["Lx"], job["Ly"], job["Lz"], job["J"], job["H1"], job["T"], job["seed"],
               y_mode=job["y_mode"], replica=job["replica"])
    o.set_spins(spins)
    o.sweep_count = sweep
    return o.measure()


def test_film_8_full_run():
    job = WL.film_8()
    g = ig.Film(job["Lx"], job["Ly"], job["Lz"], job["J"], job["H1"], job["T"], job["seed"])
    g.init(job["init_kind"])
    g.sweep(job["n_sweeps"], job["measure_every"])
    recs = g.read_series()
    o, want = _oracle(job, job["n_sweeps"], job["measure_every"])
    assert recs.shape == (10000, 13)
    assert np.array_equal(recs, want)
    assert np.array_equal(g.get_spins(), o.get_spins())
    g.close()


def test_integration_set_full_sizes():
    jobs = WL.ti_batch(n_sweeps=3)
    b = ig.Batch(jobs)
    b.set_shape(ig.SHAPE_GRID_2)
    b.sweep(3)
    for i, j in enumerate(jobs):
        recs = b.read_series(i)
        if i < 8:  # two films of each size: spins and records
            o, want = _oracle(j, 3, 1)
            assert np.array_equal(recs, want), i
            assert np.array_equal(b.get_spins(i), o.get_spins()), i
        else:
            assert recs.shape == (3, 5 + j["Lx"])
            assert np.array_equal(recs[-1], _measured(j, b.get_spins(i), 3)), i
    b.close()


def test_temperature_scan_extremes():
    jobs = WL.t_scan_40(n_sweeps=2)
    pick = [jobs[0], jobs[-1]]
    b = ig.Batch(pick)
    b.sweep(2)
    for i, j in enumerate(pick):
        o, want = _oracle(j, 2, 1)
        assert np.array_equal(b.read_series(i), want), j["T"]
        assert np.array_equal(b.get_spins(i), o.get_spins()), j["T"]
    b.close()


def test_temperature_scan_records_of_the_whole_set():
    """All 40 films in one batch (the benchmark's launch): for every fourth
    film, its last record is the oracle's measurement of its final spins."""
    jobs = WL.t_scan_40(n_sweeps=3)
    b = ig.Batch(jobs)
    b.sweep(3)
    for i in range(0, len(jobs), 4):
        recs = b.read_series(i)
        assert recs.shape == (3, 5 + jobs[i]["Lx"])
        assert np.array_equal(recs[-1], _measured(jobs[i], b.get_spins(i), 3)), jobs[i]["T"]
    b.close()


def test_job_stream_shapes_through_the_server():
    jobs = WL.serve_2000()[:24]
    for j in jobs:
        j["n_sweeps"] = 12
        j["measure_every"] = 3
    srv = ig.Server(2 << 30, chunk_sweeps=5)
    tickets = srv.submit(jobs)
    for t, j in zip(tickets, jobs):
        srv.wait(t, 600.0)
        recs, spins, _ = srv.result(t)
        o, want = _oracle(j, 12, 3)
        assert np.array_equal(recs, want), t
        assert np.array_equal(spins, o.get_spins()), t
    srv.close()
