"""The paper's measurement procedures on the GPU path.

Each procedure runs its whole film set (``workloads.*_set``) as one batch,
meaning shared launches across films of mixed size and boundary, captured in
CUDA graphs.  Its reduction is one library call over the films' record
series (``ising_procedure_*``): the exact integer means, the per-site
normalisations and the FP64 analysis all run there; this module only sorts
the series by role and marshals them.

  contact_angle       Secs. II B, III A: theta(H1) from the dividing plane
                      (Eqs. 17-18), the Young difference (Eq. 9), Young's
                      angle (Eq. 8) and gamma(theta) (Eq. 16)
  interface_tension   Sec. II C: dF = F_APBC - F_PBC by beta integration
                      (Eq. 19), then gamma(pi/2) and tau(0, pi/2) (Eq. 20)
  line_tension        Sec. IV: the residual of Eq. 21 per size and its
                      slope in Lz over a constant-area set
  stiffness_and_steps Secs. III B, III C: Eqs. 23-24, 26 and the step model
"""
from __future__ import annotations

import ctypes as _c

import numpy as np

from .binding import Batch, IsingSeries, check, lib


def run(workload, use_graph=True, autotune=True):
    """All films of the set in one batch (the library's default lanes), its
    launch shape autotuned unless autotune is False and its record rings
    sized for the whole run; returns one record series per film.  The
    records do not depend on the shape or the lanes."""
    b = Batch(workload["jobs"])
    try:
        if autotune:
            b.autotune()
        b.reserve_records(workload["n_sweeps"])
        b.sweep(workload["n_sweeps"], use_graph)
        return [b.read_series(i) for i in range(len(workload["jobs"]))]
    finally:
        b.close()


class _Series:
    """ising_series arrays over chosen films (keeps the record arrays alive)."""

    def __init__(self, records, jobs, picks):
        self.keep = [np.ascontiguousarray(records[i], dtype=np.int64) for i in picks]
        self.arr = (IsingSeries * max(len(picks), 1))()
        for k, (i, r) in enumerate(zip(picks, self.keep)):
            j = jobs[i]
            self.arr[k] = IsingSeries(r.ctypes.data, r.shape[0], int(j["Lx"]), int(j["Ly"]), int(j["Lz"]),
                                      float(j.get("J", 1.0)), float(j.get("H", 0.0)), float(j["H1"]))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(_c.c_void_p)


def _index(wl):
    return {role: i for i, role in enumerate(wl["roles"])}


def contact_angle(wl, records, gamma_pi2):
    at, k, n_gl = _index(wl), len(wl["H1s"]), wl["n_gl"]
    inter = _Series(records, wl["jobs"], [at[("interface", j)] for j in range(k)])
    plus = _Series(records, wl["jobs"], [at[("plus", j)] for j in range(k)])
    node = _Series(records, wl["jobs"], [at[("node", j, i)] for j in range(k) for i in range(n_gl)])
    H1 = _f64(wl["H1s"])
    theta, young, delta_f1, gamma = (np.zeros(k) for _ in range(4))
    y_plus = np.zeros((k, wl["Lx"]))
    check(lib().ising_procedure_contact_angle(k, _p(H1), n_gl, inter.arr, plus.arr, node.arr, int(wl["first"]),
                                              float(gamma_pi2), _p(theta), _p(young), _p(delta_f1), _p(gamma),
                                              _p(y_plus)), "ising_procedure_contact_angle")
    return dict(H1=H1, theta=theta, theta_young=young, delta_f1=delta_f1, gamma=gamma, y_plus=y_plus)


def interface_tension(wl, records):
    at, sizes, betas = _index(wl), wl["sizes"], _f64(wl["betas"])
    ns, nb = len(sizes), len(betas)
    apbc = _Series(records, wl["jobs"], [at[("apbc", s, b)] for s in range(ns) for b in range(nb)])
    pbc = _Series(records, wl["jobs"], [at[("pbc", s, b)] for s in range(ns) for b in range(nb)])
    L = _f64(sizes)
    dF = np.zeros(ns)
    g, t = _c.c_double(), _c.c_double()
    check(lib().ising_procedure_interface_tension(ns, _p(L), nb, _p(betas), apbc.arr, pbc.arr, int(wl["first"]),
                                                  _p(dF), _c.byref(g), _c.byref(t)),
          "ising_procedure_interface_tension")
    return dict(sizes=L, dF=dF, gamma_pi2=g.value, tau0=t.value)


def line_tension(wl, records, theta, gamma_theta, gamma_pi2):
    at, ns, n_gl = _index(wl), len(wl["sizes"]), wl["n_gl"]
    inter = _Series(records, wl["jobs"], [at[("interface", s, i)] for s in range(ns) for i in range(n_gl)])
    plus = _Series(records, wl["jobs"], [at[("plus", s, i)] for s in range(ns) for i in range(n_gl)])
    R, dF_film, s_wall, delta_f1 = (np.zeros(ns) for _ in range(4))
    dtau, intercept = _c.c_double(), _c.c_double()
    check(lib().ising_procedure_line_tension(ns, n_gl, float(wl["H1"]), inter.arr, plus.arr, int(wl["first"]),
                                             float(theta), float(gamma_theta), float(gamma_pi2), _p(R),
                                             _p(dF_film), _p(s_wall), _p(delta_f1), _c.byref(dtau),
                                             _c.byref(intercept)), "ising_procedure_line_tension")
    Lz = np.array([v[2] for v in wl["sizes"]], dtype=np.float64)
    return dict(Lz=Lz, R=R, dF_film=dF_film, s_wall=s_wall, delta_f1=delta_f1, dtau=dtau.value,
                intercept=intercept.value)


def stiffness_and_steps(theta, gamma, gamma_pi2, T, Lx, Lz, H1s):
    """Eqs. 23-24 and 26 from gamma(theta); Eqs. 28-32 at the measured f_s."""
    th, g, h = _f64(theta), _f64(gamma), _f64(H1s)
    phi = np.zeros(h.size)
    c, kappa, f_s, flat, h1s = (_c.c_double() for _ in range(5))
    check(lib().ising_procedure_stiffness_steps(th.size, _p(th), _p(g), float(gamma_pi2), float(T), float(Lx),
                                                float(Lz), h.size, _p(h), _c.byref(c), _c.byref(kappa),
                                                _c.byref(f_s), _c.byref(flat), _p(phi), _c.byref(h1s)),
          "ising_procedure_stiffness_steps")
    return dict(c=c.value, kappa=kappa.value, f_s=f_s.value, gamma_flat=flat.value, phi=phi, h1_star=h1s.value)
