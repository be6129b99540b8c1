"""Bulk critical point of the oracle's dynamics (slow statistical pin).

With periodic x and y, H = H1 = 0, the film is the simple-cubic Ising model.
The Binder cumulant U4 = 1 - <M^4> / (3 <M^2>^2) of cubes of edge L = 8 and
L = 16 must cross near k_B T_c / J = 4.5115 (beta_c ~ 0.2217, Fig. 7): below
T_c the larger cube has the larger U4, above it the smaller one.  The chains
run on all host cores in a spawn pool (processes started before any GPU use).
"""
import math
import multiprocessing as mp
import os

import numpy as np
import pytest

TC = 4.5115
T_LO, T_HI = 4.49, 4.53


def _chain(args):
    L, T, seed, n_eq, n_meas = args
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    from oracle import oracle as O
    O.set_threads(1)
    f = O.Film(L, L, L, 1.0, 0.0, T, seed, y_mode=O.Y_PBC, x_mode=O.X_PBC)
    f.init(O.INIT_ALL_UP)
    f.sweep(n_eq)
    M = f.sweep(n_meas, 2)[:, 2].astype(np.float64) / L ** 3
    return L, T, M


def _u4_with_error(series_list, nbins=20):
    """U4 and its jackknife error over bins of the pooled chains."""
    bins = []
    for M in series_list:
        n = (M.size // nbins) * nbins
        for b in M[:n].reshape(nbins, -1):
            bins.append(((b ** 2).mean(), (b ** 4).mean()))
    bins = np.array(bins)
    m2, m4 = bins[:, 0].mean(), bins[:, 1].mean()
    u = 1 - m4 / (3 * m2 ** 2)
    jk = []
    for i in range(len(bins)):
        rest = np.delete(bins, i, axis=0)
        a2, a4 = rest[:, 0].mean(), rest[:, 1].mean()
        jk.append(1 - a4 / (3 * a2 ** 2))
    jk = np.array(jk)
    err = math.sqrt((len(jk) - 1) * ((jk - jk.mean()) ** 2).mean())
    return u, err


@pytest.mark.slow
def test_binder_cumulant_crossing_near_tc():
    ncpu = max(2, min(os.cpu_count() or 2, 8))
    reps16 = max(1, ncpu // 2)
    jobs = []
    for T in (T_LO, T_HI):
        for r in range(reps16):
            jobs.append((16, T, 1000 + r, 1500, 60000))
        jobs.append((8, T, 2000, 2000, 200000))
    ctx = mp.get_context("spawn")
    with ctx.Pool(ncpu) as pool:
        out = pool.map(_chain, jobs)
    u = {}
    for T in (T_LO, T_HI):
        for L in (8, 16):
            u[(L, T)] = _u4_with_error([M for (l, t, M) in out if l == L and t == T])
    d_lo = u[(16, T_LO)][0] - u[(8, T_LO)][0]
    d_hi = u[(16, T_HI)][0] - u[(8, T_HI)][0]
    e_lo = math.hypot(u[(16, T_LO)][1], u[(8, T_LO)][1])
    e_hi = math.hypot(u[(16, T_HI)][1], u[(8, T_HI)][1])
    # ordered side: larger cube more ordered; disordered side: the reverse
    assert d_lo > 3 * e_lo, (u, d_lo, e_lo)
    assert d_hi < -3 * e_hi, (u, d_hi, e_hi)
    # linear interpolation of the difference locates the crossing
    t_cross = T_LO + (T_HI - T_LO) * d_lo / (d_lo - d_hi)
    dt = (T_HI - T_LO) * math.hypot(e_lo * d_hi, e_hi * d_lo) / (d_lo - d_hi) ** 2
    assert abs(t_cross - TC) < max(4 * dt, 0.015), (t_cross, dt)
