"""Ising-film oracle — TEST INFRASTRUCTURE ONLY.

ctypes wrapper around ``ising_oracle.c`` (the plain CPU simulator of the
checkerboard Metropolis sweep of Eq. 1 with the boundary rules of Sec. II A
and Eq. 11) plus the host-side thermodynamic-integration arithmetic the paper
applies to its outputs (Eqs. 9 and 19), written independently of the product.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of
``bench.py`` may import this module.  It never imports the product package.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ising_oracle.c")
LIB = os.path.join(HERE, "_build", "libising_oracle.so")

Y_GAPBC, Y_PBC, Y_APBC = 0, 1, 2
X_FREE, X_PBC = 0, 1
INIT_RANDOM, INIT_SLAB_Y, INIT_ALL_UP = 0, 1, 2

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math: exp/floor/ldexp must be libm's)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.c_void_p
            L.orc_create.restype = P
            L.orc_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_uint64]
            L.orc_set_options.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint32]
            L.orc_destroy.argtypes = [P]
            L.orc_set_spins.argtypes = [P, P]
            L.orc_get_spins.argtypes = [P, P]
            L.orc_set_sweep.argtypes = [P, ctypes.c_uint64]
            L.orc_get_sweep.argtypes = [P]
            L.orc_get_sweep.restype = ctypes.c_uint64
            L.orc_init.argtypes = [P, ctypes.c_int, ctypes.c_double]
            L.orc_sweep.argtypes = [P, ctypes.c_uint64, ctypes.c_uint32, P, ctypes.c_int64]
            L.orc_sweep.restype = ctypes.c_int64
            L.orc_measure.argtypes = [P, P]
            L.orc_energy.argtypes = [P]
            L.orc_energy.restype = ctypes.c_double
            L.orc_delta_e.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.orc_delta_e.restype = ctypes.c_double
            L.orc_accept.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_uint32]
            L.orc_philox4x32_10_n.argtypes = [P, P, P, ctypes.c_int64]
            L.orc_set_threads.argtypes = [ctypes.c_int]
            L.orc_get_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def philox4x32_10(ctrs, key):
    """Philox4x32-10 of an (n, 4) uint32 counter array under a 2-word key."""
    c = np.ascontiguousarray(np.asarray(ctrs, dtype=np.uint32).reshape(-1, 4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.empty_like(c)
    lib().orc_philox4x32_10_n(c.ctypes.data, k.ctypes.data, out.ctypes.data, c.shape[0])
    return out


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


class Film:
    """One Lx x Ly x Lz film simulated by the oracle (int8 spins, canonical
    order ((kx-1)*Ly + (ky-1))*Lz + (kz-1))."""

    def __init__(self, Lx, Ly, Lz, J=1.0, H1=0.0, T=3.0, seed=1, *, y_mode=Y_GAPBC,
                 x_mode=X_FREE, H=0.0, replica=0):
        self.Lx, self.Ly, self.Lz = int(Lx), int(Ly), int(Lz)
        self.J, self.H1, self.T, self.H = float(J), float(H1), float(T), float(H)
        self._h = lib().orc_create(self.Lx, self.Ly, self.Lz, self.J, self.H1, self.T, int(seed))
        if not self._h:
            raise ValueError("invalid film parameters")
        if lib().orc_set_options(self._h, int(y_mode), int(x_mode), self.H, int(replica)) != 0:
            raise ValueError("invalid options")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    @property
    def n_sites(self):
        return self.Lx * self.Ly * self.Lz

    @property
    def record_len(self):
        return 5 + self.Lx

    def init(self, kind=INIT_RANDOM, flip_p=0.0):
        if lib().orc_init(self._h, int(kind), float(flip_p)) != 0:
            raise ValueError("bad init")

    def set_spins(self, s):
        a = np.ascontiguousarray(np.asarray(s, dtype=np.int8).reshape(-1))
        assert a.size == self.n_sites
        lib().orc_set_spins(self._h, a.ctypes.data)

    def get_spins(self):
        a = np.empty(self.n_sites, dtype=np.int8)
        lib().orc_get_spins(self._h, a.ctypes.data)
        return a

    @property
    def sweep_count(self):
        return int(lib().orc_get_sweep(self._h))

    @sweep_count.setter
    def sweep_count(self, v):
        lib().orc_set_sweep(self._h, int(v))

    def sweep(self, n, measure_every=0):
        """Run n sweeps; returns the (n_records, 5+Lx) int64 records."""
        n = int(n)
        cap = n // measure_every + 1 if measure_every else 0
        recs = np.zeros((max(cap, 1), self.record_len), dtype=np.int64)
        got = lib().orc_sweep(self._h, n, int(measure_every), recs.ctypes.data if cap else None, cap)
        if got < 0:
            raise ValueError("sweep counter exhausted")
        return recs[:got]

    def measure(self):
        rec = np.zeros(self.record_len, dtype=np.int64)
        lib().orc_measure(self._h, rec.ctypes.data)
        return rec

    def energy(self):
        return float(lib().orc_energy(self._h))

    def delta_e(self, kx, ky, kz):
        return float(lib().orc_delta_e(self._h, kx, ky, kz))


def accept(dE, T, u) -> bool:
    return bool(lib().orc_accept(float(dE), float(T), int(u)))


def energy_from_record(rec, J, H, H1):
    """Eq. 1 from one record's integers: E = -J B - H M - H1 M1 - Hn Mn, Hn = -H1."""
    return -J * float(rec[1]) - H * float(rec[2]) - H1 * float(rec[3]) - (-H1) * float(rec[4])
