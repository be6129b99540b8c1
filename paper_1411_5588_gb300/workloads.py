"""Seeded synthetic workloads shaped like the paper's runs.

Plain data only (film shapes, temperatures, fields, seeds, sweep counts,
arrival times): nothing here performs any step of the Monte Carlo method.
Both the CUDA path and the CPU oracle are driven from these lists.

  film_8      8^3 film, T = 3, H1 = +0.5, Eq. 11 boundary, random start, seed 1
  film_46m    120 x 240 x 1600 film (46,080,000 spins; stands in for the
              paper's 184 x 504 x 504 lattices), T = 3, H1 = +0.55, slab start
              along y with 1% flips, seed 2, records every 10 sweeps
  ti_batch    64 films: 16 Gauss-Legendre nodes of H1 in [0, 0.75] x T in
              {2.0, 3.5} x seeds {1, 2}; Lx in {32, 48, 64, 96} by replica
              index, Ly = 2 Lx, Lz = 4 Lx; random start; records every sweep
  serve_2000  2000 jobs, Poisson arrivals at 200 jobs/s, each axis drawn
              log-uniformly (Lx 16..96, Ly 16..192, Lz 16..768, Lz even), T
              uniform in [1.5, 4.2], H1 uniform in [0, 1], sweeps log-uniform
              in [500, 5000], seed 3
  t_scan_40   40 films 120 x 240 x 1600 at T = 1.5 .. 4.4 (step 0.0744),
              H1 = 0.55, slab start (seed 5), records every sweep
"""
from __future__ import annotations

import numpy as np

Y_GAPBC, INIT_RANDOM, INIT_SLAB_Y = 0, 0, 1


def film_8():
    return dict(Lx=8, Ly=8, Lz=8, J=1.0, H1=0.5, T=3.0, seed=1, replica=0, y_mode=Y_GAPBC,
                init_kind=INIT_RANDOM, flip_p=0.0, measure_every=1, n_sweeps=10000)


def film_46m(replica=0):
    return dict(Lx=120, Ly=240, Lz=1600, J=1.0, H1=0.55, T=3.0, seed=2, replica=replica, y_mode=Y_GAPBC,
                init_kind=INIT_SLAB_Y, flip_p=0.01, measure_every=10, n_sweeps=2000)


def ti_batch(n_sweeps=5000):
    t, _ = np.polynomial.legendre.leggauss(16)
    nodes = 0.375 * (t + 1.0)  # H1 in [0, 0.75]
    jobs = []
    for node in range(16):
        for ti, T in enumerate((2.0, 3.5)):
            for si, seed in enumerate((1, 2)):
                r = (node * 2 + ti) * 2 + si
                Lx = (32, 48, 64, 96)[r % 4]
                jobs.append(dict(Lx=Lx, Ly=2 * Lx, Lz=4 * Lx, J=1.0, H1=float(nodes[node]), T=T, seed=seed,
                                 replica=r, y_mode=Y_GAPBC, init_kind=INIT_RANDOM, flip_p=0.0, measure_every=1,
                                 n_sweeps=n_sweeps))
    return jobs


def _loguniform(rng, lo, hi, size):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size))


def serve_2000(n_jobs=2000, rate=200.0, seed=3, measure_every=10):
    rng = np.random.Generator(np.random.Philox(seed))
    gaps = rng.exponential(1.0 / rate, n_jobs)
    arrival = np.cumsum(gaps) - gaps[0]
    Lx = np.rint(_loguniform(rng, 16, 96, n_jobs)).astype(int)
    Ly = np.rint(_loguniform(rng, 16, 192, n_jobs)).astype(int)
    Lz = np.rint(_loguniform(rng, 16, 768, n_jobs)).astype(int)
    Lz += Lz % 2
    T = rng.uniform(1.5, 4.2, n_jobs)
    H1 = rng.uniform(0.0, 1.0, n_jobs)
    sweeps = np.rint(_loguniform(rng, 500, 5000, n_jobs)).astype(int)
    jobs = []
    for i in range(n_jobs):
        jobs.append(dict(Lx=int(Lx[i]), Ly=int(Ly[i]), Lz=int(Lz[i]), J=1.0, H1=float(H1[i]), T=float(T[i]),
                         seed=seed, replica=i, y_mode=Y_GAPBC, init_kind=INIT_RANDOM, flip_p=0.0,
                         measure_every=measure_every, n_sweeps=int(sweeps[i]), arrival=float(arrival[i])))
    return jobs


def t_scan_40(n_sweeps=10000):
    temps = 1.5 + 0.0744 * np.arange(40)
    return [dict(Lx=120, Ly=240, Lz=1600, J=1.0, H1=0.55, T=float(T), seed=5, replica=i, y_mode=Y_GAPBC,
                 init_kind=INIT_SLAB_Y, flip_p=0.01, measure_every=1, n_sweeps=n_sweeps)
            for i, T in enumerate(temps)]


def sites(job):
    return int(job["Lx"]) * int(job["Ly"]) * int(job["Lz"])
