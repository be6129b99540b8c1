"""The paper's measurement procedures on the GPU path.

Each procedure runs its whole film set (``workloads.*_set``) as one batch,
meaning shared launches across films of mixed size and boundary, captured in
CUDA graphs. It then reduces the int64 records with the library's exact
integer means and FP64 analysis calls.

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

import math

import numpy as np

from . import analysis as A
from .binding import Batch, series_energy, series_mean, ti_surface_field


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


def _wall_means(rec, job, first):
    """Per-site layer-1 and layer-Lx magnetisations (records columns 3, 4)."""
    area = job["Ly"] * job["Lz"]
    return series_mean(rec, 3, first) / area, series_mean(rec, 4, first) / area


def contact_angle(wl, records, gamma_pi2):
    first, Lx, Ly, Lz = wl["first"], wl["Lx"], wl["Ly"], wl["Lz"]
    H1s = wl["H1s"]
    k = len(H1s)
    inter, plus = [None] * k, [None] * k
    m1 = [[None] * wl["n_gl"] for _ in range(k)]
    mn = [[None] * wl["n_gl"] for _ in range(k)]
    for rec, job, role in zip(records, wl["jobs"], wl["roles"]):
        if role[0] == "interface":
            inter[role[1]] = rec
        elif role[0] == "plus":
            plus[role[1]] = rec
        else:
            m1[role[1]][role[2]], mn[role[1]][role[2]] = _wall_means(rec, job, first)
    theta, young, delta_f1, y_plus = [], [], [], []
    for j, h in enumerate(H1s):
        mbar = A.layer_profile(inter[j], Lx, Ly, Lz, first)
        m_plus = A.layer_profile(plus[j], Lx, Ly, Lz, first)
        th, yp = A.contact_angle(Ly, mbar, m_plus, A.mirror_profile(m_plus))
        d = A.ti_young_difference(h, m1[j], mn[j])
        theta.append(th)
        y_plus.append(yp)
        delta_f1.append(d)
        young.append(A.young_angle(d, gamma_pi2) if abs(d) <= gamma_pi2 else float("nan"))
    # Eq. 16 from the perpendicular interface at H1 = 0
    th_path = np.concatenate([[math.pi / 2], theta])
    df_path = np.concatenate([[0.0], np.abs(delta_f1)])
    gamma = A.gamma_of_theta(th_path, df_path, gamma_pi2)[1:]
    return dict(H1=np.array(H1s), theta=np.array(theta), theta_young=np.array(young),
                delta_f1=np.array(delta_f1), gamma=gamma, y_plus=np.array(y_plus))


def interface_tension(wl, records):
    first, betas, sizes = wl["first"], np.asarray(wl["betas"]), wl["sizes"]
    U = {}
    for rec, job, role in zip(records, wl["jobs"], wl["roles"]):
        U[role] = series_energy(rec, job["J"], job["H1"], first=first)[1]  # <E> of Eq. 1
    dF = []
    for s, L in enumerate(sizes):
        dU = np.array([U[("apbc", s, k)] - U[("pbc", s, k)] for k in range(len(betas))])
        dF.append(A.ti_free_energy_beta(betas, dU, 0.0)[-1])
    L = np.array(sizes, dtype=np.float64)
    gamma_pi2, tau0 = A.fit_gamma_tau(L, L, dF)
    return dict(sizes=L, dF=np.array(dF), gamma_pi2=gamma_pi2, tau0=tau0)


def line_tension(wl, records, theta, gamma_theta, gamma_pi2):
    first, H1, n = wl["first"], wl["H1"], wl["n_gl"]
    sizes = wl["sizes"]
    M1 = [[None] * n for _ in sizes]
    Mn = [[None] * n for _ in sizes]
    m1 = [[None] * n for _ in sizes]
    mn = [[None] * n for _ in sizes]
    for rec, job, role in zip(records, wl["jobs"], wl["roles"]):
        s, i = role[1], role[2]
        if role[0] == "interface":
            M1[s][i], Mn[s][i] = series_mean(rec, 3, first), series_mean(rec, 4, first)
        else:
            m1[s][i], mn[s][i] = _wall_means(rec, job, first)
    R, dF_film, s_wall, delta_f1 = [], [], [], []
    for s, (Lx, Ly, Lz) in enumerate(sizes):
        dF = ti_surface_field(H1, M1[s], Mn[s])  # totals: F_int(H1) - F_int(0)
        sw = ti_surface_field(H1, m1[s], mn[s])  # per wall site
        df1 = A.ti_young_difference(H1, m1[s], mn[s])
        R.append(A.line_tension_residual(dF, Lx, Ly, Lz, theta, gamma_theta, gamma_pi2, sw, df1))
        dF_film.append(dF)
        s_wall.append(sw)
        delta_f1.append(df1)
    Lz = np.array([v[2] for v in sizes], dtype=np.float64)
    dtau, intercept = A.line_tension_lz_scan(Lz, R)
    return dict(Lz=Lz, R=np.array(R), dF_film=np.array(dF_film), s_wall=np.array(s_wall),
                delta_f1=np.array(delta_f1), dtau=dtau, intercept=intercept)


def stiffness_and_steps(theta, gamma, gamma_pi2, T, Lx, Lz, H1s):
    """Eqs. 23-24 and 26 from gamma(theta); Eqs. 28-32 at the measured f_s."""
    c, kappa = A.stiffness(theta, gamma, gamma_pi2)
    th = np.concatenate([[math.pi / 2], theta])
    g = np.concatenate([[gamma_pi2], gamma])
    f_s, gamma_flat = A.step_free_energy(th, g)
    model = [A.step_model(h, f_s, T, Lx, Lz) for h in H1s]
    return dict(c=c, kappa=kappa, f_s=f_s, gamma_flat=gamma_flat, phi=np.array([m[0] for m in model]),
                h1_star=model[0][1])
