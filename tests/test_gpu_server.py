"""Continuous-batching server: every job's records and final spins equal the
oracle's chain for that job alone, whatever else shares the device; the
arena budget forces queueing; waits are bounded."""
import time

import numpy as np
import pytest

import paper_1411_5588_gb300 as ig
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _specs():
    shapes = [(8, 8, 8), (6, 10, 34), (16, 16, 16), (4, 6, 130), (12, 5, 64), (3, 3, 2), (10, 20, 40),
              (7, 7, 70), (5, 9, 96), (16, 8, 32), (2, 4, 256), (9, 6, 12)]
    out = []
    for i, (Lx, Ly, Lz) in enumerate(shapes):
        out.append(dict(Lx=Lx, Ly=Ly, Lz=Lz, T=1.5 + 0.25 * i, H1=0.08 * i, seed=3, replica=i,
                        measure_every=(i % 4) + 1, n_sweeps=37 + 13 * i,
                        init_kind=[ig.INIT_RANDOM, ig.INIT_SLAB_Y, ig.INIT_ALL_UP][i % 3], flip_p=0.01,
                        y_mode=[ig.Y_GAPBC, ig.Y_PBC, ig.Y_APBC][i % 3]))
    return out


def _oracle(sp):
    o = O.Film(sp["Lx"], sp["Ly"], sp["Lz"], 1.0, sp["H1"], sp["T"], sp["seed"], y_mode=sp["y_mode"],
               replica=sp["replica"])
    o.init(sp["init_kind"], sp["flip_p"])
    recs = o.sweep(sp["n_sweeps"], sp["measure_every"])
    return recs, o.get_spins()


@pytest.mark.parametrize("budget,chunk,cold", [(64 << 20, 16, False), (1 << 20, 7, False), (64 << 20, 11, True)])
def test_server_jobs_match_oracle(budget, chunk, cold):
    """cold: a T -> 0 job (exact-table kernel while it is resident) and a
    beta = 0 job in the stream."""
    specs = _specs()
    if cold:
        specs[3]["T"] = 1e-3
        specs[7]["T"] = float("inf")
    srv = ig.Server(budget, chunk_sweeps=chunk)
    tickets = srv.submit(specs[:5])
    tickets += srv.submit(specs[5:])
    for t, sp in zip(tickets, specs):
        srv.wait(t, 300.0)
        recs, spins, info = srv.result(t)
        want_r, want_s = _oracle(sp)
        assert np.array_equal(recs, want_r), t
        assert np.array_equal(spins, want_s), t
        assert info["t_submit"] <= info["t_admit"] <= info["t_finish"]
    st = srv.stats()
    assert st["finished"] == len(specs) and st["running"] == 0 and st["queued"] == 0
    assert st["bytes_in_use"] == 0
    srv.close()


def test_server_wait_times_out_and_rejects_oversize():
    srv = ig.Server(1 << 20, chunk_sweeps=50)
    with pytest.raises(ig.IsingError) as e:
        srv.submit([dict(Lx=128, Ly=128, Lz=128, T=3.0, n_sweeps=10)])  # staging alone exceeds 1 MiB
    assert e.value.status == ig.EINVAL
    (t,) = srv.submit([dict(Lx=16, Ly=16, Lz=32, T=3.0, n_sweeps=20000, measure_every=0)])
    with pytest.raises(ig.IsingError) as e:
        srv.wait(t, 0.0)
    assert e.value.status == ig.ETIMEOUT
    with pytest.raises(ig.IsingError) as e:
        srv.result(t)
    assert e.value.status == ig.EBUSY
    srv.wait(t, 300.0)
    srv.result(t, want_spins=False)
    srv.close()


def test_late_job_shares_chunks_with_a_running_job():
    """Continuous batching, not a queue: a job submitted while another is on
    the device is admitted at the next chunk boundary and runs in the same
    launches (their chunk ranges intersect, and it is admitted before the
    first job finishes).  A server that ran jobs one after another would give
    the second job a first chunk after the first job's last.  Both results
    are still the oracle's chains for each job alone."""
    long_job = dict(Lx=8, Ly=8, Lz=16, T=2.5, H1=0.3, seed=11, replica=0, measure_every=100, n_sweeps=20000,
                    init_kind=ig.INIT_RANDOM, flip_p=0.0, y_mode=ig.Y_GAPBC)
    late_job = dict(Lx=6, Ly=10, Lz=34, T=3.5, H1=0.2, seed=11, replica=1, measure_every=7, n_sweeps=300,
                    init_kind=ig.INIT_SLAB_Y, flip_p=0.01, y_mode=ig.Y_GAPBC)
    srv = ig.Server(64 << 20, chunk_sweeps=50)
    (ta,) = srv.submit([long_job])
    deadline = time.monotonic() + 60.0
    while srv.stats()["chunks"] < 2:  # the long job is on the device
        assert time.monotonic() < deadline
        time.sleep(0.0005)
    assert not srv.poll(ta)
    (tb,) = srv.submit([late_job])
    srv.wait(tb, 300.0)
    srv.wait(ta, 300.0)
    ra, sa, ia = srv.result(ta)
    rb, sb, ib = srv.result(tb)
    assert ib["first_chunk"] > ia["first_chunk"]
    assert ib["first_chunk"] <= ib["last_chunk"] <= ia["last_chunk"]  # ran inside the long job's chunks
    assert ib["t_admit"] < ia["t_finish"] and ib["t_finish"] <= ia["t_finish"]
    for (recs, spins), sp in (((ra, sa), long_job), ((rb, sb), late_job)):
        want_r, want_s = _oracle(sp)
        assert np.array_equal(recs, want_r)
        assert np.array_equal(spins, want_s)
    srv.close()


def test_single_sweep_jobs_and_zero_sweep_jobs():
    """The smallest jobs: one sweep, recorded or not, beside a long one and
    inside one chunk; they finish in the first chunk and still equal the
    oracle's chain alone.  A job of no sweeps is refused at submission."""
    base = dict(Lx=6, Ly=7, Lz=18, T=2.7, H1=0.3, seed=4, init_kind=ig.INIT_SLAB_Y, flip_p=0.02,
                y_mode=ig.Y_GAPBC)
    specs = [dict(base, replica=0, n_sweeps=1, measure_every=1),
             dict(base, replica=1, n_sweeps=1, measure_every=0),
             dict(base, replica=2, n_sweeps=90, measure_every=4),
             dict(base, replica=3, n_sweeps=1, measure_every=2)]
    srv = ig.Server(64 << 20, chunk_sweeps=16)
    with pytest.raises(ig.IsingError) as e:
        srv.submit([dict(base, replica=9, n_sweeps=0)])
    assert e.value.status == ig.EINVAL
    tickets = srv.submit(specs)
    for t, sp in zip(tickets, specs):
        srv.wait(t, 300.0)
        recs, spins, info = srv.result(t)
        want_r, want_s = _oracle(sp)
        assert recs.shape == want_r.shape, t
        assert np.array_equal(recs, want_r), t
        assert np.array_equal(spins, want_s), t
        if sp["n_sweeps"] == 1:
            assert info["first_chunk"] == info["last_chunk"], t
    srv.close()
