"""The paper's measurement procedures on the oracle -- TEST INFRASTRUCTURE ONLY.

The same film sets as the product's procedures (a workload dict: film list
and roles, passed in by the caller). Each film is run one at a time by the
CPU simulator, and the records are reduced with oracle/analysis.py and
oracle/ti.py. It shares no code with the product and imports nothing from it.

  contact_angle       Secs. II B, III A (Eqs. 8, 9, 12, 16-18)
  interface_tension   Sec. II C (Eqs. 19-20)
  line_tension        Sec. IV (Eqs. 21-22)
  stiffness_and_steps Secs. III B, III C (Eqs. 23-24, 26, 28-32)

The composition (which films feed which terms, which record columns, the
per-site normalisations, the integration limits) is pinned on hand-built
records whose reductions have closed forms (tests/test_oracle_workflows.py).
"""
from __future__ import annotations

import math

import numpy as np

from . import analysis as OA
from . import oracle as O
from . import ti as OT


def run(workload):
    out = []
    for job in workload["jobs"]:
        f = O.Film(job["Lx"], job["Ly"], job["Lz"], job["J"], job["H1"], job["T"], job["seed"],
                   y_mode=job["y_mode"], replica=job["replica"])
        f.init(job["init_kind"], job["flip_p"])
        out.append(f.sweep(workload["n_sweeps"], job["measure_every"]))
    return out


def _walls(rec, job, first):
    area = job["Ly"] * job["Lz"]
    return OT.series_mean(rec, 3, first) / area, OT.series_mean(rec, 4, first) / area


def contact_angle(wl, records, gamma_pi2):
    first, Lx, Ly, Lz, H1s = wl["first"], wl["Lx"], wl["Ly"], wl["Lz"], wl["H1s"]
    by_role = {role: (rec, job) for rec, job, role in zip(records, wl["jobs"], wl["roles"])}
    out = dict(H1=np.array(H1s), theta=[], theta_young=[], delta_f1=[], y_plus=[])
    for j, h in enumerate(H1s):
        mbar = OA.layer_profile(by_role[("interface", j)][0], Lx, Ly, Lz, first)
        mp = OA.layer_profile(by_role[("plus", j)][0], Lx, Ly, Lz, first)
        th, yp = OA.contact_angle(Ly, mbar, mp, OA.mirror_profile(mp))
        walls = [_walls(*by_role[("node", j, i)], first) for i in range(wl["n_gl"])]
        d = OA.ti_young_difference(h, [w[0] for w in walls], [w[1] for w in walls])
        out["theta"].append(th)
        out["y_plus"].append(yp)
        out["delta_f1"].append(d)
        out["theta_young"].append(OA.young_angle(d, gamma_pi2) if abs(d) <= gamma_pi2 else float("nan"))
    gamma = OA.gamma_of_theta([math.pi / 2] + out["theta"], [0.0] + [abs(d) for d in out["delta_f1"]], gamma_pi2)
    out["gamma"] = gamma[1:]
    return {k: np.asarray(v) for k, v in out.items()}


def interface_tension(wl, records):
    first, betas = wl["first"], np.asarray(wl["betas"])
    U = {role: OT.series_energy_mean(rec, job["J"], 0.0, job["H1"], first)
         for rec, job, role in zip(records, wl["jobs"], wl["roles"])}
    dF = []
    for s, _ in enumerate(wl["sizes"]):
        dU = [U[("apbc", s, k)] - U[("pbc", s, k)] for k in range(len(betas))]
        dF.append(OA.ti_free_energy_beta(betas, dU, 0.0)[-1])
    L = np.array(wl["sizes"], dtype=np.float64)
    g, t = OA.fit_gamma_tau(L, L, dF)
    return dict(sizes=L, dF=np.array(dF), gamma_pi2=g, tau0=t)


def line_tension(wl, records, theta, gamma_theta, gamma_pi2):
    first, H1, n = wl["first"], wl["H1"], wl["n_gl"]
    by_role = {role: (rec, job) for rec, job, role in zip(records, wl["jobs"], wl["roles"])}
    out = dict(R=[], dF_film=[], s_wall=[], delta_f1=[])
    for s, (Lx, Ly, Lz) in enumerate(wl["sizes"]):
        M1 = [OT.series_mean(by_role[("interface", s, i)][0], 3, first) for i in range(n)]
        Mn = [OT.series_mean(by_role[("interface", s, i)][0], 4, first) for i in range(n)]
        walls = [_walls(*by_role[("plus", s, i)], first) for i in range(n)]
        m1, mn = [w[0] for w in walls], [w[1] for w in walls]
        dF = OT.surface_field_ti(H1, M1, Mn)
        sw = OT.surface_field_ti(H1, m1, mn)
        df1 = OA.ti_young_difference(H1, m1, mn)
        out["R"].append(OA.line_tension_residual(dF, Lx, Ly, Lz, theta, gamma_theta, gamma_pi2, sw, df1))
        out["dF_film"].append(dF)
        out["s_wall"].append(sw)
        out["delta_f1"].append(df1)
    Lz = np.array([v[2] for v in wl["sizes"]], dtype=np.float64)
    dtau, intercept = OA.line_tension_lz_scan(Lz, out["R"])
    res = {k: np.asarray(v) for k, v in out.items()}
    res.update(Lz=Lz, dtau=dtau, intercept=intercept)
    return res


def stiffness_and_steps(theta, gamma, gamma_pi2, T, Lx, Lz, H1s):
    c, kappa = OA.stiffness(theta, gamma, gamma_pi2)
    f_s, gamma_flat = OA.step_free_energy([math.pi / 2] + list(theta), [gamma_pi2] + list(gamma))
    model = [OA.step_model(h, f_s, T, Lx, Lz) for h in H1s]
    return dict(c=c, kappa=kappa, f_s=f_s, gamma_flat=gamma_flat, phi=np.array([m[0] for m in model]),
                h1_star=model[0][1])
