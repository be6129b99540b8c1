"""ctypes binding of ``include/ising.h`` (argument marshalling only).

Every function of the C ABI is available under its own name on ``lib()``;
``Film``, ``Batch`` and ``Server`` wrap the handles.  All computation happens
in the CUDA library ``_build/libising_gb300.so``; there is no fallback: if the
library is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libising_gb300.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EBUSY, ENOTFOUND = range(7)
Y_GAPBC, Y_PBC, Y_APBC = 0, 1, 2
X_FREE, X_PBC = 0, 1
INIT_RANDOM, INIT_SLAB_Y, INIT_ALL_UP = 0, 1, 2
SHAPE_AUTO, SHAPE_RESIDENT, SHAPE_GRID_1, SHAPE_GRID_2, SHAPE_GRID_Q, SHAPE_CLUSTER = 0, 1, 2, 3, 4, 5
MAX_LANES = 16  # ISING_MAX_LANES

_c = ctypes
P = _c.c_void_p
I8P = _c.POINTER(_c.c_int8)
I64P = _c.POINTER(_c.c_int64)
U32P = _c.POINTER(_c.c_uint32)
DP = _c.POINTER(_c.c_double)


class IsingObs(_c.Structure):
    _fields_ = [("sweep", _c.c_uint64), ("bond_sum", _c.c_int64), ("M", _c.c_int64), ("M1", _c.c_int64),
                ("Mn", _c.c_int64), ("m_x", I64P)]


class IsingJob(_c.Structure):
    _fields_ = [("Lx", _c.c_int32), ("Ly", _c.c_int32), ("Lz", _c.c_int32), ("y_mode", _c.c_int32),
                ("x_mode", _c.c_int32), ("init_kind", _c.c_int32), ("J", _c.c_double), ("H", _c.c_double),
                ("H1", _c.c_double), ("T", _c.c_double), ("flip_p", _c.c_double), ("seed", _c.c_uint64),
                ("replica", _c.c_uint32), ("measure_every", _c.c_uint32), ("n_sweeps", _c.c_uint64)]


class IsingJobInfo(_c.Structure):
    _fields_ = [("t_submit", _c.c_double), ("t_admit", _c.c_double), ("t_finish", _c.c_double),
                ("n_records", _c.c_uint64), ("first_chunk", _c.c_uint64), ("last_chunk", _c.c_uint64)]


class IsingSeries(_c.Structure):
    _fields_ = [("records", P), ("n", _c.c_size_t), ("Lx", _c.c_int), ("Ly", _c.c_int), ("Lz", _c.c_int),
                ("J", _c.c_double), ("H", _c.c_double), ("H1", _c.c_double)]


class IsingServerStats(_c.Structure):
    _fields_ = [("bytes_in_use", _c.c_size_t), ("bytes_budget", _c.c_size_t), ("queued", _c.c_uint64),
                ("running", _c.c_uint64), ("finished", _c.c_uint64), ("chunks", _c.c_uint64),
                ("attempts", _c.c_uint64)]


_SIGS = {
    "ising_create": [_c.c_int, _c.c_int, _c.c_int, _c.c_double, _c.c_double, _c.c_double, _c.c_uint64,
                     _c.POINTER(P)],
    "ising_set_options": [P, _c.c_int, _c.c_int, _c.c_double, _c.c_uint32],
    "ising_set_shape": [P, _c.c_int],
    "ising_reserve_records": [P, _c.c_uint64],
    "ising_read_series_async": [P, P, _c.c_size_t, _c.POINTER(_c.c_size_t), P],
    "ising_batch_reserve_records": [P, _c.c_uint64],
    "ising_get_shape": [P, _c.c_uint32, _c.POINTER(_c.c_int)],
    "ising_autotune": [P, _c.c_uint32, _c.POINTER(_c.c_int)],
    "ising_batch_set_shape": [P, _c.c_int],
    "ising_batch_get_shape": [P, _c.POINTER(_c.c_int)],
    "ising_batch_set_cluster_size": [P, _c.c_uint32],
    "ising_batch_get_cluster_size": [P, U32P],
    "ising_batch_autotune": [P, _c.POINTER(_c.c_int)],
    "ising_set_params": [P, _c.c_double, _c.c_double, _c.c_double],
    "ising_set_stream": [P, P],
    "ising_init": [P, _c.c_int, _c.c_double],
    "ising_set_spins": [P, P],
    "ising_get_spins": [P, P],
    "ising_set_spins_device": [P, P],
    "ising_get_spins_device": [P, P],
    "ising_packed_words": [P],
    "ising_get_packed_device": [P, P],
    "ising_set_packed_device": [P, P],
    "ising_get_sweep": [P, _c.POINTER(_c.c_uint64)],
    "ising_set_sweep": [P, _c.c_uint64],
    "ising_sweep": [P, _c.c_uint64, _c.c_uint32],
    "ising_measure": [P, _c.POINTER(IsingObs)],
    "ising_read_series": [P, P, _c.c_size_t, _c.POINTER(_c.c_size_t)],
    "ising_pending_records": [P, _c.POINTER(_c.c_size_t)],
    "ising_synchronize": [P, _c.c_double],
    "ising_destroy": [P],
    "ising_batch_create": [_c.POINTER(IsingJob), _c.c_size_t, _c.POINTER(P)],
    "ising_batch_create_lanes": [_c.POINTER(IsingJob), _c.c_size_t, _c.c_uint32, _c.POINTER(P)],
    "ising_batch_get_lanes": [P, _c.POINTER(_c.c_uint32)],
    "ising_batch_set_stream": [P, P],
    "ising_batch_sweep": [P, _c.c_uint64, _c.c_int],
    "ising_batch_get_spins": [P, _c.c_size_t, P],
    "ising_batch_read_series": [P, _c.c_size_t, P, _c.c_size_t, _c.POINTER(_c.c_size_t)],
    "ising_batch_synchronize": [P, _c.c_double],
    "ising_batch_pending_records": [P, _c.c_size_t, _c.POINTER(_c.c_size_t)],
    "ising_batch_destroy": [P],
    "ising_server_create": [_c.c_size_t, _c.c_uint32, _c.POINTER(P)],
    "ising_batch_submit": [P, _c.POINTER(IsingJob), _c.c_size_t, _c.POINTER(_c.c_uint64)],
    "ising_batch_poll": [P, _c.c_uint64, _c.POINTER(_c.c_int)],
    "ising_batch_wait": [P, _c.c_uint64, _c.c_double],
    "ising_batch_result": [P, _c.c_uint64, P, _c.c_size_t, P, _c.POINTER(IsingJobInfo)],
    "ising_server_get_stats": [P, _c.POINTER(IsingServerStats)],
    "ising_server_destroy": [P],
    "ising_gauss_legendre": [_c.c_int, _c.c_double, _c.c_double, P, P],
    "ising_series_mean": [P, _c.c_size_t, _c.c_size_t, _c.c_size_t, _c.c_size_t, DP],
    "ising_ti_surface_field": [_c.c_int, _c.c_double, P, P, DP],
    "ising_series_energy": [P, _c.c_size_t, _c.c_int, _c.c_double, _c.c_double, _c.c_double, P, _c.c_size_t, DP],
    "ising_ti_beta_trapezoid": [_c.c_int, P, P, DP],
    "ising_ti_temperature_trapezoid": [_c.c_int, P, P, DP],
    "ising_ti_young_difference": [_c.c_int, _c.c_double, P, P, DP],
    "ising_layer_profile": [P, _c.c_size_t, _c.c_int, _c.c_int, _c.c_int, _c.c_size_t, P],
    "ising_mirror_profile": [_c.c_int, P, P],
    "ising_contact_angle": [_c.c_int, _c.c_int, P, P, P, _c.c_int, _c.c_int, P, DP],
    "ising_young_angle": [_c.c_double, _c.c_double, DP],
    "ising_gamma_of_theta": [_c.c_int, P, P, _c.c_double, P],
    "ising_ti_free_energy_beta": [_c.c_int, P, P, _c.c_double, P],
    "ising_fit_gamma_tau": [_c.c_int, P, P, P, DP, DP],
    "ising_line_tension_residual": [_c.c_double] * 9 + [DP],
    "ising_line_tension_lz_scan": [_c.c_int, P, P, DP, DP],
    "ising_stiffness": [_c.c_int, P, P, _c.c_double, DP, DP],
    "ising_roughening_kappa_fit": [_c.c_int, P, P, _c.c_double, _c.c_double, DP],
    "ising_step_free_energy": [_c.c_int, P, P, DP, DP],
    "ising_roughening_fs_fit": [_c.c_int, P, P, _c.c_double, DP, DP],
    "ising_step_model": [_c.c_double] * 5 + [DP, DP],
    "ising_critical_field": [_c.c_int, P, P] + [_c.c_double] * 4 + [DP, DP],
    "ising_procedure_contact_angle": [_c.c_int, P, _c.c_int, P, P, P, _c.c_size_t, _c.c_double, P, P, P, P, P],
    "ising_procedure_interface_tension": [_c.c_int, P, _c.c_int, P, P, P, _c.c_size_t, P, DP, DP],
    "ising_procedure_line_tension": [_c.c_int, _c.c_int, _c.c_double, P, P, _c.c_size_t, _c.c_double, _c.c_double,
                                     _c.c_double, P, P, P, P, DP, DP],
    "ising_procedure_stiffness_steps": [_c.c_int, P, P, _c.c_double, _c.c_double, _c.c_double, _c.c_double,
                                        _c.c_int, P, DP, DP, DP, DP, P, DP],
    "ising_measure_packed_noalloc": [P, _c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_uint64, P, P],
    "ising_check_counters": [_c.POINTER(_c.c_int), _c.POINTER(_c.c_uint64), _c.POINTER(_c.c_uint64)],
    "ising_strerror": [_c.c_int],
    "ising_last_error": [],
    "ising_version": [_c.POINTER(_c.c_int), _c.POINTER(_c.c_int), _c.POINTER(_c.c_int)],
}
_RESTYPE = {"ising_strerror": _c.c_char_p, "ising_last_error": _c.c_char_p, "ising_packed_words": _c.c_size_t}

_lock = threading.Lock()
_lib = None


class IsingError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = lib().ising_last_error().decode(errors="replace")
        super().__init__(f"{where}: {lib().ising_strerror(status).decode()} ({status}): {msg}")


def lib():
    """Load the CUDA library (building it first if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                from . import build as _build
                _build.build()
            L = ctypes.CDLL(LIB_PATH)
            for name, args in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = _RESTYPE.get(name, _c.c_int)
            _lib = L
    return _lib


def check(status, where):
    if status != OK:
        raise IsingError(status, where)


def _ptr(a):
    return a.ctypes.data_as(P)


def _torch_stream(stream):
    if stream is None:
        return None
    return P(int(getattr(stream, "cuda_stream", stream)))


class Film:
    """One film (``ising_create`` ... ``ising_destroy``)."""

    def __init__(self, Lx, Ly, Lz, J=1.0, H1=0.0, T=3.0, seed=1, *, y_mode=Y_GAPBC, x_mode=X_FREE, H=0.0,
                 replica=0, stream=None, shape=SHAPE_AUTO):
        self.Lx, self.Ly, self.Lz = int(Lx), int(Ly), int(Lz)
        self.J, self.H1, self.T, self.H = float(J), float(H1), float(T), float(H)
        h = P()
        check(lib().ising_create(self.Lx, self.Ly, self.Lz, self.J, self.H1, self.T, int(seed), _c.byref(h)),
              "ising_create")
        self._h = h
        check(lib().ising_set_options(h, int(y_mode), int(x_mode), self.H, int(replica)), "ising_set_options")
        if stream is not None:
            check(lib().ising_set_stream(h, _torch_stream(stream)), "ising_set_stream")
        if shape != SHAPE_AUTO:
            self.set_shape(shape)

    def set_shape(self, shape):
        check(lib().ising_set_shape(self._h, int(shape)), "ising_set_shape")

    def reserve_records(self, n):
        check(lib().ising_reserve_records(self._h, int(n)), "ising_reserve_records")

    def read_series_async(self, host_ptr, cap, stream=None):
        """Enqueue the copy of up to cap pending records to host memory at
        host_ptr (pinned, (cap, 5 + Lx) int64) on stream (torch stream or
        None for the handle's copy stream); returns the count."""
        n = _c.c_size_t()
        s = _torch_stream(stream) if stream is not None else None
        check(lib().ising_read_series_async(self._h, P(int(host_ptr)), int(cap), _c.byref(n), s),
              "ising_read_series_async")
        return n.value

    def get_shape(self, measure_every):
        v = _c.c_int()
        check(lib().ising_get_shape(self._h, int(measure_every), _c.byref(v)), "ising_get_shape")
        return v.value

    def autotune(self, measure_every):
        """Time every launch shape on a scratch film; returns the fastest."""
        v = _c.c_int()
        check(lib().ising_autotune(self._h, int(measure_every), _c.byref(v)), "ising_autotune")
        return v.value

    def close(self):
        if getattr(self, "_h", None):
            lib().ising_destroy(self._h)
            self._h = None

    __del__ = close

    @property
    def n_sites(self):
        return self.Lx * self.Ly * self.Lz

    @property
    def record_len(self):
        return 5 + self.Lx

    def set_params(self, J, H1, T):
        self.J, self.H1, self.T = float(J), float(H1), float(T)
        check(lib().ising_set_params(self._h, self.J, self.H1, self.T), "ising_set_params")

    def set_stream(self, stream):
        check(lib().ising_set_stream(self._h, _torch_stream(stream)), "ising_set_stream")

    def init(self, kind=INIT_RANDOM, flip_p=0.0):
        check(lib().ising_init(self._h, int(kind), float(flip_p)), "ising_init")

    def set_spins(self, s):
        a = np.ascontiguousarray(np.asarray(s, dtype=np.int8).reshape(-1))
        if a.size != self.n_sites:
            raise ValueError("wrong number of spins")
        check(lib().ising_set_spins(self._h, _ptr(a)), "ising_set_spins")

    def get_spins(self):
        a = np.empty(self.n_sites, dtype=np.int8)
        check(lib().ising_get_spins(self._h, _ptr(a)), "ising_get_spins")
        return a

    def set_spins_device(self, ptr):
        check(lib().ising_set_spins_device(self._h, P(int(ptr))), "ising_set_spins_device")

    def get_spins_device(self, ptr):
        check(lib().ising_get_spins_device(self._h, P(int(ptr))), "ising_get_spins_device")

    def packed_words(self):
        return int(lib().ising_packed_words(self._h))

    def get_packed_device(self, ptr):
        check(lib().ising_get_packed_device(self._h, P(int(ptr))), "ising_get_packed_device")

    def set_packed_device(self, ptr):
        check(lib().ising_set_packed_device(self._h, P(int(ptr))), "ising_set_packed_device")

    @property
    def sweep_count(self):
        v = _c.c_uint64()
        check(lib().ising_get_sweep(self._h, _c.byref(v)), "ising_get_sweep")
        return int(v.value)

    @sweep_count.setter
    def sweep_count(self, v):
        check(lib().ising_set_sweep(self._h, int(v)), "ising_set_sweep")

    def sweep(self, n, measure_every=0):
        """Enqueue n sweeps (asynchronous)."""
        check(lib().ising_sweep(self._h, int(n), int(measure_every)), "ising_sweep")

    def measure(self):
        m = np.zeros(self.Lx, dtype=np.int64)
        o = IsingObs()
        o.m_x = m.ctypes.data_as(I64P)
        check(lib().ising_measure(self._h, _c.byref(o)), "ising_measure")
        return np.concatenate([[o.sweep, o.bond_sum, o.M, o.M1, o.Mn], m]).astype(np.int64)

    def pending_records(self):
        n = _c.c_size_t()
        check(lib().ising_pending_records(self._h, _c.byref(n)), "ising_pending_records")
        return int(n.value)

    def read_series(self, cap=None):
        if cap is None:
            cap = self.pending_records()
        buf = np.zeros((max(cap, 1), self.record_len), dtype=np.int64)
        n = _c.c_size_t()
        check(lib().ising_read_series(self._h, _ptr(buf), int(cap), _c.byref(n)), "ising_read_series")
        return buf[: n.value]

    def synchronize(self, timeout_s=600.0):
        check(lib().ising_synchronize(self._h, float(timeout_s)), "ising_synchronize")


def make_jobs(specs):
    """Array of IsingJob from dicts (missing keys take defaults)."""
    arr = (IsingJob * len(specs))()
    for i, sp in enumerate(specs):
        j = arr[i]
        j.Lx, j.Ly, j.Lz = int(sp["Lx"]), int(sp["Ly"]), int(sp["Lz"])
        j.y_mode = int(sp.get("y_mode", Y_GAPBC))
        j.x_mode = int(sp.get("x_mode", X_FREE))
        j.init_kind = int(sp.get("init_kind", INIT_RANDOM))
        j.J = float(sp.get("J", 1.0))
        j.H = float(sp.get("H", 0.0))
        j.H1 = float(sp.get("H1", 0.0))
        j.T = float(sp["T"])
        j.flip_p = float(sp.get("flip_p", 0.0))
        j.seed = int(sp.get("seed", 1))
        j.replica = int(sp.get("replica", 0))
        j.measure_every = int(sp.get("measure_every", 0))
        j.n_sweeps = int(sp.get("n_sweeps", 0))
    return arr


class Batch:
    """Films updated by shared launches (``ising_batch_*``), spread over
    ``lanes`` concurrent lanes (0: the library's default)."""

    def __init__(self, specs, stream=None, lanes=0):
        self.specs = [dict(s) for s in specs]
        self._jobs = make_jobs(self.specs)
        h = P()
        check(lib().ising_batch_create_lanes(self._jobs, len(self.specs), int(lanes), _c.byref(h)),
              "ising_batch_create_lanes")
        self._h = h
        if stream is not None:
            check(lib().ising_batch_set_stream(h, _torch_stream(stream)), "ising_batch_set_stream")

    def close(self):
        if getattr(self, "_h", None):
            lib().ising_batch_destroy(self._h)
            self._h = None

    __del__ = close

    def __len__(self):
        return len(self.specs)

    @property
    def lanes(self):
        v = _c.c_uint32()
        check(lib().ising_batch_get_lanes(self._h, _c.byref(v)), "ising_batch_get_lanes")
        return int(v.value)

    def sweep(self, n, use_graph=False):
        check(lib().ising_batch_sweep(self._h, int(n), 1 if use_graph else 0), "ising_batch_sweep")

    def set_shape(self, shape):
        check(lib().ising_batch_set_shape(self._h, int(shape)), "ising_batch_set_shape")

    def reserve_records(self, n):
        check(lib().ising_batch_reserve_records(self._h, int(n)), "ising_batch_reserve_records")

    def get_shape(self):
        v = _c.c_int()
        check(lib().ising_batch_get_shape(self._h, _c.byref(v)), "ising_batch_get_shape")
        return v.value

    def set_cluster_size(self, cluster_size):
        """CTAs per film of the CLUSTER shape (0: automatic)."""
        check(lib().ising_batch_set_cluster_size(self._h, int(cluster_size)), "ising_batch_set_cluster_size")

    @property
    def cluster_size(self):
        v = _c.c_uint32()
        check(lib().ising_batch_get_cluster_size(self._h, _c.byref(v)), "ising_batch_get_cluster_size")
        return int(v.value)

    def autotune(self):
        """Time the grid shapes and the cluster sizes on a scratch batch; adopts and returns the fastest."""
        v = _c.c_int()
        check(lib().ising_batch_autotune(self._h, _c.byref(v)), "ising_batch_autotune")
        return v.value

    def get_spins(self, i):
        s = self.specs[i]
        a = np.empty(int(s["Lx"]) * int(s["Ly"]) * int(s["Lz"]), dtype=np.int8)
        check(lib().ising_batch_get_spins(self._h, int(i), _ptr(a)), "ising_batch_get_spins")
        return a

    def pending_records(self, i):
        n = _c.c_size_t()
        check(lib().ising_batch_pending_records(self._h, int(i), _c.byref(n)), "ising_batch_pending_records")
        return n.value

    def read_series(self, i, cap=None):
        rl = 5 + int(self.specs[i]["Lx"])
        if cap is None:
            cap = self.pending_records(i)
        buf = np.zeros((max(cap, 1), rl), dtype=np.int64)
        n = _c.c_size_t()
        check(lib().ising_batch_read_series(self._h, int(i), _ptr(buf), int(cap), _c.byref(n)),
              "ising_batch_read_series")
        return buf[: n.value]

    def synchronize(self, timeout_s=600.0):
        check(lib().ising_batch_synchronize(self._h, float(timeout_s)), "ising_batch_synchronize")


class Server:
    """Continuous-batching server (``ising_server_*`` / ``ising_batch_submit``...)."""

    def __init__(self, hbm_budget_bytes, chunk_sweeps=100):
        h = P()
        check(lib().ising_server_create(int(hbm_budget_bytes), int(chunk_sweeps), _c.byref(h)),
              "ising_server_create")
        self._h = h
        self._specs = {}

    def close(self):
        if getattr(self, "_h", None):
            lib().ising_server_destroy(self._h)
            self._h = None

    __del__ = close

    def submit(self, specs):
        jobs = make_jobs(specs)
        first = _c.c_uint64()
        check(lib().ising_batch_submit(self._h, jobs, len(specs), _c.byref(first)), "ising_batch_submit")
        tickets = [first.value + i for i in range(len(specs))]
        for t, s in zip(tickets, specs):
            self._specs[t] = dict(s)
        return tickets

    def poll(self, t):
        d = _c.c_int()
        check(lib().ising_batch_poll(self._h, int(t), _c.byref(d)), "ising_batch_poll")
        return bool(d.value)

    def wait(self, t, timeout_s=600.0):
        check(lib().ising_batch_wait(self._h, int(t), float(timeout_s)), "ising_batch_wait")

    def result(self, t, want_spins=True):
        s = self._specs[t]
        rl = 5 + int(s["Lx"])
        m = int(s.get("measure_every", 0))
        nrec = int(s["n_sweeps"]) // m if m else 0
        buf = np.zeros((max(nrec, 1), rl), dtype=np.int64)
        spins = np.empty(int(s["Lx"]) * int(s["Ly"]) * int(s["Lz"]), dtype=np.int8) if want_spins else None
        info = IsingJobInfo()
        check(lib().ising_batch_result(self._h, int(t), _ptr(buf), nrec, _ptr(spins) if want_spins else None,
                                       _c.byref(info)), "ising_batch_result")
        del self._specs[t]
        return buf[:nrec], spins, {"t_submit": info.t_submit, "t_admit": info.t_admit, "t_finish": info.t_finish,
                                   "n_records": int(info.n_records), "first_chunk": int(info.first_chunk),
                                   "last_chunk": int(info.last_chunk)}

    def stats(self):
        st = IsingServerStats()
        check(lib().ising_server_get_stats(self._h, _c.byref(st)), "ising_server_get_stats")
        return {k: getattr(st, k) for k, _ in IsingServerStats._fields_}


# ------------------------------------------------------------- host FP64

def check_counters():
    """(checked build?, out-of-range accesses so far, the first one)."""
    c, n, f = _c.c_int(), _c.c_uint64(), _c.c_uint64()
    check(lib().ising_check_counters(_c.byref(c), _c.byref(n), _c.byref(f)), "ising_check_counters")
    return bool(c.value), n.value, f.value


def gauss_legendre(n, a, b):
    x = np.zeros(n)
    w = np.zeros(n)
    check(lib().ising_gauss_legendre(int(n), float(a), float(b), _ptr(x), _ptr(w)), "ising_gauss_legendre")
    return x, w


def series_mean(records, col, first=0):
    r = np.ascontiguousarray(records, dtype=np.int64)
    out = _c.c_double()
    check(lib().ising_series_mean(_ptr(r), r.shape[0], r.shape[1], int(col), int(first), _c.byref(out)),
          "ising_series_mean")
    return out.value


def series_energy(records, J, H1, H=0.0, first=0):
    """Eq. 1 per record and the mean over records[first:] (exact integer sums)."""
    r = np.ascontiguousarray(records, dtype=np.int64)
    E = np.zeros(r.shape[0])
    mean = _c.c_double()
    check(lib().ising_series_energy(_ptr(r), r.shape[0], r.shape[1] - 5, float(J), float(H), float(H1), _ptr(E),
                                    int(first), _c.byref(mean)), "ising_series_energy")
    return E, mean.value


def ti_surface_field(H1, m1, mn):
    m1 = np.ascontiguousarray(m1, dtype=np.float64)
    mn = np.ascontiguousarray(mn, dtype=np.float64)
    out = _c.c_double()
    check(lib().ising_ti_surface_field(m1.size, float(H1), _ptr(m1), _ptr(mn), _c.byref(out)),
          "ising_ti_surface_field")
    return out.value


def ti_beta_trapezoid(beta, U):
    b = np.ascontiguousarray(beta, dtype=np.float64)
    u = np.ascontiguousarray(U, dtype=np.float64)
    out = _c.c_double()
    check(lib().ising_ti_beta_trapezoid(b.size, _ptr(b), _ptr(u), _c.byref(out)), "ising_ti_beta_trapezoid")
    return out.value


def ti_temperature_trapezoid(T, U):
    t = np.ascontiguousarray(T, dtype=np.float64)
    u = np.ascontiguousarray(U, dtype=np.float64)
    out = _c.c_double()
    check(lib().ising_ti_temperature_trapezoid(t.size, _ptr(t), _ptr(u), _c.byref(out)),
          "ising_ti_temperature_trapezoid")
    return out.value
