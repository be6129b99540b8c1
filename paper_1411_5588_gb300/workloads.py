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

The three film sets of the paper's procedures (Secs. II B, II C, III, IV);
``roles`` tags each film with what it measures:
  contact_angle_set     per H1: the film with the Eq. 11 boundary from a
                        slab start ("interface"), a periodic-y film from all
                        up ("plus", the (+) plateaus), and periodic-y films at
                        n_gl Gauss-Legendre nodes of [0, H1] ("node")
  interface_tension_set per size Lx = Lz and per beta on a grid from 0.2:
                        antiperiodic ("apbc") and periodic ("pbc") y, H1 = 0
                        (default sizes: Fig. 12's Lx = Lz = 20..50, Ly = 60)
  line_tension_set      per size of a constant-area set (Lx Lz and Ly Lz
                        fixed): films with the Eq. 11 boundary ("interface")
                        and periodic-y films ("plus") at the nodes of [0, H1]
                        (default: Fig. 13's Lx Lz = 1536, Ly Lz = 9216 with
                        Lz = 16..96 at H1 = 0.45)
"""
from __future__ import annotations

import numpy as np

Y_GAPBC, Y_PBC, Y_APBC = 0, 1, 2
INIT_RANDOM, INIT_SLAB_Y, INIT_ALL_UP = 0, 1, 2


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


def _nodes(n, a, b):
    t, _ = np.polynomial.legendre.leggauss(int(n))
    return 0.5 * (b - a) * (t + 1.0) + a


def _film(Lx, Ly, Lz, T, H1, seed, replica, y_mode, init_kind, n_sweeps):
    return dict(Lx=int(Lx), Ly=int(Ly), Lz=int(Lz), J=1.0, H1=float(H1), T=float(T), seed=int(seed),
                replica=int(replica), y_mode=y_mode, init_kind=init_kind, flip_p=0.0, measure_every=1,
                n_sweeps=int(n_sweeps))


def contact_angle_set(Lx=32, Ly=96, Lz=64, T=3.0, H1s=(0.15, 0.3, 0.45, 0.55), n_gl=8, n_sweeps=2000,
                      first=500, seed=7):
    jobs, roles = [], []
    for j, h in enumerate(H1s):
        jobs.append(_film(Lx, Ly, Lz, T, h, seed, len(jobs), Y_GAPBC, INIT_SLAB_Y, n_sweeps))
        roles.append(("interface", j))
        jobs.append(_film(Lx, Ly, Lz, T, h, seed, len(jobs), Y_PBC, INIT_ALL_UP, n_sweeps))
        roles.append(("plus", j))
        for i, x in enumerate(_nodes(n_gl, 0.0, h)):
            jobs.append(_film(Lx, Ly, Lz, T, x, seed, len(jobs), Y_PBC, INIT_ALL_UP, n_sweeps))
            roles.append(("node", j, i))
    return dict(kind="contact_angle", Lx=Lx, Ly=Ly, Lz=Lz, T=T, H1s=tuple(float(h) for h in H1s), n_gl=n_gl,
                n_sweeps=n_sweeps, first=first, jobs=jobs, roles=roles)


def interface_tension_set(sizes=(20, 30, 40, 50), Ly=60, T=3.0, beta0=0.2, n_beta=24, n_sweeps=2000, first=500,
                          seed=8):
    betas = np.linspace(beta0, 1.0 / T, n_beta)
    jobs, roles = [], []
    for s, L in enumerate(sizes):
        for k, b in enumerate(betas):
            for name, mode in (("apbc", Y_APBC), ("pbc", Y_PBC)):
                jobs.append(_film(L, Ly, L, 1.0 / b, 0.0, seed, len(jobs), mode, INIT_ALL_UP, n_sweeps))
                roles.append((name, s, k))
    return dict(kind="interface_tension", sizes=tuple(sizes), Ly=Ly, T=T, betas=betas, n_sweeps=n_sweeps,
                first=first, jobs=jobs, roles=roles)


def line_tension_set(sizes=((96, 576, 16), (48, 288, 32), (32, 192, 48), (24, 144, 64), (16, 96, 96)), T=3.0,
                     H1=0.45, n_gl=8, n_sweeps=2000, first=500, seed=9):
    jobs, roles = [], []
    for s, (Lx, Ly, Lz) in enumerate(sizes):
        for i, x in enumerate(_nodes(n_gl, 0.0, H1)):
            jobs.append(_film(Lx, Ly, Lz, T, x, seed, len(jobs), Y_GAPBC, INIT_SLAB_Y, n_sweeps))
            roles.append(("interface", s, i))
            jobs.append(_film(Lx, Ly, Lz, T, x, seed, len(jobs), Y_PBC, INIT_ALL_UP, n_sweeps))
            roles.append(("plus", s, i))
    return dict(kind="line_tension", sizes=tuple(tuple(v) for v in sizes), T=T, H1=float(H1), n_gl=n_gl,
                n_sweeps=n_sweeps, first=first, jobs=jobs, roles=roles)
