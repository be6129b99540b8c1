"""Exact reference computations used to pin the oracle (test code only).

Everything here is written independently of ``oracle/ising_oracle.c``: the
film's bonds are listed explicitly from 0-based coordinates, the Boltzmann
sums are done by brute-force enumeration of all 2^N states, and the one-sweep
transition matrix is assembled from that bond list.  A mistake in the oracle's
neighbour rules, field terms, schedule or acceptance rule therefore shows up as
a disagreement with these numbers.
"""
from __future__ import annotations

import math

import numpy as np

Y_GAPBC, Y_PBC, Y_APBC = 0, 1, 2


def site_index(Lx, Ly, Lz, x, y, z):
    """0-based coordinates -> canonical index ((kx-1)*Ly + (ky-1))*Lz + (kz-1)."""
    return (x * Ly + y) * Lz + z


def bond_list(Lx, Ly, Lz, y_mode=Y_GAPBC, x_pbc=False):
    """Every bond of the film once, as (i, j, sign).

    x: free surfaces (or periodic when x_pbc); z: periodic; y: the last row
    y = Ly-1 couples to row 0 -- through the reflected layer Lx-1-x with a
    minus sign for the generalized antiperiodic rule (Eq. 11), the same layer
    with a plus sign (PBC) or a minus sign (APBC).  A wrap that lands on the
    same neighbour as an interior bond (Lz = 2, Ly = 2, Lx = 2 periodic) is a
    second bond between the pair.
    """
    out = []
    for x in range(Lx):
        for y in range(Ly):
            for z in range(Lz):
                i = site_index(Lx, Ly, Lz, x, y, z)
                # +x
                if x + 1 < Lx:
                    out.append((i, site_index(Lx, Ly, Lz, x + 1, y, z), 1))
                elif x_pbc:
                    out.append((i, site_index(Lx, Ly, Lz, 0, y, z), 1))
                # +y
                if y + 1 < Ly:
                    out.append((i, site_index(Lx, Ly, Lz, x, y + 1, z), 1))
                elif y_mode == Y_GAPBC:
                    out.append((i, site_index(Lx, Ly, Lz, Lx - 1 - x, 0, z), -1))
                elif y_mode == Y_PBC:
                    out.append((i, site_index(Lx, Ly, Lz, x, 0, z), 1))
                else:
                    out.append((i, site_index(Lx, Ly, Lz, x, 0, z), -1))
                # +z
                out.append((i, site_index(Lx, Ly, Lz, x, y, (z + 1) % Lz), 1))
    return np.array(out, dtype=np.int64).reshape(-1, 3)


def layer_fields(Lx, H, H1):
    """Field on each layer: H everywhere, +H1 on the first, Hn = -H1 on the last."""
    h = np.full(Lx, float(H))
    h[0] += H1
    h[Lx - 1] += -H1
    return h


def configs_pm1(N):
    """All 2^N spin configurations as an int8 (2^N, N) array of +-1."""
    states = np.arange(1 << N, dtype=np.int64)
    bits = (states[:, None] >> np.arange(N, dtype=np.int64)[None, :]) & 1
    return (1 - 2 * bits).astype(np.int8)


def observables(S, Lx, Ly, Lz, bonds):
    """Bond sum B, M, layer sums m(x) for configurations S (n, N)."""
    S = np.asarray(S, dtype=np.int64)
    B = np.zeros(S.shape[0], dtype=np.int64)
    for i, j, sg in bonds:
        B += sg * S[:, i] * S[:, j]
    m = S.reshape(S.shape[0], Lx, Ly * Lz).sum(axis=2)
    return B, m.sum(axis=1), m


def energies(S, Lx, Ly, Lz, J, H, H1, y_mode=Y_GAPBC, x_pbc=False):
    bonds = bond_list(Lx, Ly, Lz, y_mode, x_pbc)
    B, M, m = observables(S, Lx, Ly, Lz, bonds)
    h = layer_fields(Lx, H, H1)
    return -J * B - (m * h[None, :]).sum(axis=1)


def exact_averages(Lx, Ly, Lz, J, H, H1, T, y_mode=Y_GAPBC, x_pbc=False):
    """Boltzmann averages by enumeration (N <= 20)."""
    N = Lx * Ly * Lz
    assert N <= 20
    S = configs_pm1(N)
    bonds = bond_list(Lx, Ly, Lz, y_mode, x_pbc)
    B, M, m = observables(S, Lx, Ly, Lz, bonds)
    h = layer_fields(Lx, H, H1)
    E = -J * B - (m * h[None, :]).sum(axis=1)
    if math.isinf(T):
        w = np.ones_like(E)
    else:
        w = np.exp(-(E - E.min()) / T)
    w /= w.sum()
    return {
        "E": float((w * E).sum()),
        "B": float((w * B).sum()),
        "M": float((w * M).sum()),
        "absM": float((w * np.abs(M)).sum()),
        "M1": float((w * m[:, 0]).sum()),
        "Mn": float((w * m[:, Lx - 1]).sum()),
        "m": (w[:, None] * m).sum(axis=0),
        "Emin": float(E.min()),
        "Bmax": int(B.max()),
    }


# --------------------------------------------------------- transition matrix

def phases(Lx, Ly, Lz, n_phases=4):
    """Site sets of the sweep, 0-based: colour (x+y+z) % 2 of the 1-based
    coordinates equals (x+y+z+3) % 2.  Four phases: colour 0 rows y<Ly-1, colour
    0 row Ly-1, colour 1 rows y<Ly-1, colour 1 row Ly-1.  n_phases=2 gives the
    plain two-colour checkerboard (for the counter-example test)."""
    out = [[] for _ in range(n_phases)]
    for x in range(Lx):
        for y in range(Ly):
            for z in range(Lz):
                c = (x + y + z + 3) % 2
                i = site_index(Lx, Ly, Lz, x, y, z)
                if n_phases == 4:
                    out[2 * c + (1 if y == Ly - 1 else 0)].append(i)
                else:
                    out[c].append(i)
    return out


def local_fields(Lx, Ly, Lz, bonds):
    """Neighbour list with signs: nb[i] = list of (j, sign) over all slots."""
    N = Lx * Ly * Lz
    nb = [[] for _ in range(N)]
    for i, j, sg in bonds:
        nb[i].append((j, sg))
        nb[j].append((i, sg))
    return nb


def quantised_accept(dE, T):
    """Metropolis acceptance as the sweep applies it: 1 for dE <= 0, else
    floor(exp(-dE/T) * 2^32) / 2^32."""
    if dE <= 0:
        return 1.0
    p = math.exp(-dE / T)
    return math.floor(math.ldexp(p, 32)) / 2.0 ** 32


def exact_accept(dE, T):
    return 1.0 if dE <= 0 else math.exp(-dE / T)


def transition_matrix(Lx, Ly, Lz, J, H, H1, T, y_mode=Y_GAPBC, n_phases=4, acc=quantised_accept,
                      x_pbc=False):
    """One-sweep transition matrix P[s, s'] (rows: from) over all 2^N states,
    built as the product of the per-phase matrices in schedule order.  Within a
    phase each site flips independently with its Metropolis probability given
    the state at the start of the phase."""
    N = Lx * Ly * Lz
    assert N <= 12
    bonds = bond_list(Lx, Ly, Lz, y_mode, x_pbc)
    nb = local_fields(Lx, Ly, Lz, bonds)
    h = layer_fields(Lx, H, H1)
    layer = [i // (Ly * Lz) for i in range(N)]
    S = configs_pm1(N).astype(np.int64)
    nS = 1 << N
    P = np.eye(nS)
    for ph in phases(Lx, Ly, Lz, n_phases):
        Pp = np.zeros((nS, nS))
        for st in range(nS):
            s = S[st]
            probs = []
            for i in ph:
                sig = sum(sg * s[j] for j, sg in nb[i])
                dE = 2.0 * s[i] * (J * sig + h[layer[i]])
                probs.append(acc(dE, T))
            for mask in range(1 << len(ph)):
                p = 1.0
                tgt = st
                for k, i in enumerate(ph):
                    if (mask >> k) & 1:
                        p *= probs[k]
                        tgt ^= (1 << i)
                    else:
                        p *= 1.0 - probs[k]
                Pp[st, tgt] += p
        P = P @ Pp
    return P


def stationary(P):
    w, v = np.linalg.eig(P.T)
    k = int(np.argmin(np.abs(w - 1.0)))
    pi = np.real(v[:, k])
    return pi / pi.sum()


def boltzmann(Lx, Ly, Lz, J, H, H1, T, y_mode=Y_GAPBC, x_pbc=False):
    N = Lx * Ly * Lz
    E = energies(configs_pm1(N), Lx, Ly, Lz, J, H, H1, y_mode, x_pbc)
    w = np.exp(-(E - E.min()) / T)
    return w / w.sum()


def state_of(spins):
    """+-1 canonical spin vector -> enumeration index (bit i set for spin -1)."""
    s = np.asarray(spins).reshape(-1)
    return int(sum((1 << i) for i in range(s.size) if s[i] < 0))


# ------------------------------------------------------ 2D torus (Lx = 1)

def kaufman_logZ_terms(K, m, n):
    """log|Z_i| and signs of Kaufman's four products for an m x n torus
    (B. Kaufman, Phys. Rev. 76, 1232 (1949)): gamma_l from
    cosh(gamma_l) = cosh(2K) coth(2K) - cos(pi l / n), gamma_0 = 2K + ln tanh K,
    Z1 = prod_r 2cosh(m g_{2r+1}/2), Z2 = prod_r 2sinh(m g_{2r+1}/2),
    Z3 = prod_r 2cosh(m g_{2r}/2),   Z4 = prod_r 2sinh(m g_{2r}/2),
    r = 0..n-1, and the prefactor (1/2)(2 sinh 2K)^{mn/2}."""
    def gamma(l):
        if l % (2 * n) == 0:
            return 2 * K + math.log(math.tanh(K))
        return math.acosh(math.cosh(2 * K) / math.tanh(2 * K) - math.cos(math.pi * l / n))

    logs, signs = [], []
    for parity, fn in ((1, "cosh"), (1, "sinh"), (0, "cosh"), (0, "sinh")):
        lz, sg = 0.0, 1.0
        for r in range(n):
            g = gamma(2 * r + parity) * m / 2.0
            if fn == "cosh":
                lz += abs(g) + math.log1p(math.exp(-2 * abs(g)))
            else:
                if g == 0.0:
                    return None
                sg *= 1.0 if g > 0 else -1.0
                ag = abs(g)
                lz += ag + math.log1p(-math.exp(-2 * ag))
        logs.append(lz)
        signs.append(sg)
    pref = -math.log(2.0) + (m * n / 2.0) * math.log(2.0 * math.sinh(2 * K))
    return pref, logs, signs


def kaufman_logZ(K, m, n, pattern):
    """log Z = log[(1/2)(2 sinh 2K)^{mn/2} * sum_i pattern_i Z_i]."""
    pref, logs, signs = kaufman_logZ_terms(K, m, n)
    top = max(logs)
    tot = sum(p * s * math.exp(l - top) for p, s, l in zip(pattern, signs, logs))
    return pref + top + math.log(tot)


def kaufman_energy_per_bond_sum(K, m, n, pattern, dK=1e-5):
    """<B> = d log Z / dK for the m x n torus (J = 1, K = 1/T)."""
    return (kaufman_logZ(K + dK, m, n, pattern) - kaufman_logZ(K - dK, m, n, pattern)) / (2 * dK)
