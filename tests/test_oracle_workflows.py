"""Pins of the oracle's procedures (oracle/workflows.py) on hand-built
records whose reductions have closed forms: which films feed which terms,
which record columns, the per-site normalisations and the integration
limits.  The functions they call are pinned on their own in
test_oracle_analysis.py and test_ti_host.py; here only the composition is
under test, against values fixed by construction (no simulation)."""
import math

import numpy as np

from oracle import workflows as OW


def _rec(Lx, B=0, M=0, M1=0, Mn=0, m=None, n=1):
    """n identical records [sweep, B, M, M1, Mn, m(1..Lx)]."""
    r = np.zeros((n, 5 + Lx), dtype=np.int64)
    r[:, 0] = np.arange(1, n + 1)
    r[:, 1], r[:, 2], r[:, 3], r[:, 4] = B, M, M1, Mn
    if m is not None:
        r[:, 5:] = np.asarray(m, dtype=np.int64)
    return r


def test_contact_angle_workflow_on_a_planar_interface():
    """Sec. III A: plus films with m+ = 0.8 in every layer (so m- = -0.8 by
    Eq. 12) and interface films whose Eq. 18 dividing surface is the plane
    y+ = 10 + 2 kx give theta = atan(1/2); node films with m1 + mn = 0.2 give
    the Young difference -0.2 H1 (Eq. 9 is exact for constants), its angle
    by Eq. 8, and gamma(theta) by Eq. 16 integrated from gamma(pi/2)."""
    Lx, Ly, Lz, n_gl, gamma_pi2 = 8, 40, 10, 4, 0.9
    H1s = (0.15, 0.3)
    area = Ly * Lz  # 400 sites per layer
    kx = np.arange(1, Lx + 1)
    m_iface = 16 * (10 + 2 * kx) - 320  # 400 * ((10 + 2 kx) / 25 - 0.8)
    jobs, roles, records = [], [], []
    for j, _ in enumerate(H1s):
        for role, rec in ((("interface", j), _rec(Lx, m=m_iface, n=3)),
                          (("plus", j), _rec(Lx, m=np.full(Lx, 320), n=3))):
            roles.append(role)
            records.append(rec)
            jobs.append(dict(Ly=Ly, Lz=Lz))
        for i in range(n_gl):
            roles.append(("node", j, i))
            # the first record is dropped (first = 1): give it other values
            r = _rec(Lx, M1=200, Mn=-120, n=3)
            r[0, 3:5] = (-999, 999)
            records.append(r)
            jobs.append(dict(Ly=Ly, Lz=Lz))
    for r, role in zip(records, roles):
        if role[0] != "node":
            r[0, 5:] = 0  # dropped too
    wl = dict(first=1, Lx=Lx, Ly=Ly, Lz=Lz, H1s=H1s, n_gl=n_gl, jobs=jobs, roles=roles)
    out = OW.contact_angle(wl, records, gamma_pi2)
    th = math.atan(0.5)
    assert np.allclose(out["theta"], th, rtol=0, atol=1e-12)
    for yp in out["y_plus"]:
        assert np.allclose(yp, 10 + 2 * kx, rtol=0, atol=1e-12)
    d = -0.2 * np.asarray(H1s)
    assert np.allclose(out["delta_f1"], d, rtol=0, atol=1e-14)
    assert np.allclose(out["theta_young"], np.arccos(np.abs(d) / gamma_pi2), rtol=0, atol=1e-12)
    # Eq. 16 from (pi/2, gamma_pi2) over the points (pi/2, th, th): the
    # second step is empty, so both films carry the first step's value
    rhs = -np.abs(d) / math.sin(th) ** 2
    g1 = math.sin(th) * (gamma_pi2 + 0.5 * (th - math.pi / 2) * (0.0 + rhs[0]))
    assert abs(out["gamma"][0] - g1) < 1e-12


def test_interface_tension_workflow_recovers_gamma_and_tau():
    """Sec. II C: with equal wall sums in both films (so H1 = 0.25 cancels),
    bulk field H = 0 (so the films' different M does not enter) and an APBC
    film whose bond sum falls short of the PBC film's by 2 L^2 + 3 L at every
    beta, dU = J (2 L^2 + 3 L), Eq. 19
    from F(beta0) = 0 gives dF = dU (beta_end - beta0) / beta_end, and the
    Eq. 20 fit gives gamma = 2 c and tau = 1.5 c, c = J (beta_end - beta0) /
    beta_end."""
    J, sizes = 1.0, (4, 6, 8)
    betas = np.linspace(0.2, 1.0 / 3.0, 5)
    jobs, roles, records = [], [], []
    for s, L in enumerate(sizes):
        for k, _ in enumerate(betas):
            # the wall sums are the same in both films, so with H1 != 0 they
            # cancel in dU; M differs, but the bulk field H is 0
            for name, B, M in (("apbc", 3000 - (2 * L * L + 3 * L), 0), ("pbc", 3000, 400)):
                roles.append((name, s, k))
                records.append(_rec(L, B=B, M=M, M1=77, Mn=-55, n=2))
                jobs.append(dict(J=J, H1=0.25))
    wl = dict(first=0, betas=betas, sizes=sizes, jobs=jobs, roles=roles)
    out = OW.interface_tension(wl, records)
    c = J * (betas[-1] - betas[0]) / betas[-1]
    L = np.asarray(sizes, dtype=np.float64)
    assert np.allclose(out["dF"], (2 * L * L + 3 * L) * c, rtol=1e-13, atol=0)
    assert abs(out["gamma_pi2"] - 2 * c) < 1e-12 and abs(out["tau0"] - 1.5 * c) < 1e-12


def test_line_tension_workflow_feeds_each_term_from_its_films():
    """Sec. IV with the area term cancelled (gamma_theta = gamma_pi2 sin
    theta) and plus films with M1 = Mn = 0 (no wall terms): R = F_int(H1) -
    F_int(0) = -H1 (M1 - Mn) of the interface films.  Choosing M1 - Mn =
    -(8 + Lz) makes R = 4 + 0.5 Lz, so the scan gives dtau = 0.25 and
    intercept 4.  A second pass with plus-film walls m1 = 0.5, mn = -0.3
    gives s_wall = -0.8 H1 and delta_f1 = -0.2 H1 (Eq. 9)."""
    H1, n_gl, theta, gamma_pi2 = 0.5, 4, 1.2, 0.9
    gamma_theta = gamma_pi2 * math.sin(theta)
    sizes = ((12, 30, 8), (8, 45, 12), (6, 60, 16))

    def build(m1_plus, mn_plus):
        jobs, roles, records = [], [], []
        for s, (Lx, Ly, Lz) in enumerate(sizes):
            for i in range(n_gl):
                roles.append(("interface", s, i))
                records.append(_rec(Lx, M1=-(8 + Lz), Mn=0, n=2))
                jobs.append(dict(Ly=Ly, Lz=Lz))
                roles.append(("plus", s, i))
                records.append(_rec(Lx, M1=m1_plus * Ly * Lz, Mn=mn_plus * Ly * Lz, n=2))
                jobs.append(dict(Ly=Ly, Lz=Lz))
        return dict(first=0, H1=H1, n_gl=n_gl, sizes=sizes, jobs=jobs, roles=roles), records

    wl, records = build(0, 0)
    out = OW.line_tension(wl, records, theta, gamma_theta, gamma_pi2)
    Lz = np.array([s[2] for s in sizes], dtype=np.float64)
    assert np.allclose(out["dF_film"], H1 * (8 + Lz), rtol=0, atol=1e-12)
    assert np.allclose(out["R"], 4 + 0.5 * Lz, rtol=0, atol=1e-12)
    assert abs(out["dtau"] - 0.25) < 1e-12 and abs(out["intercept"] - 4.0) < 1e-11
    assert np.array_equal(out["Lz"], Lz)

    wl, records = build(0.5, -0.3)  # Ly Lz is a multiple of 10 for every size
    out = OW.line_tension(wl, records, theta, gamma_theta, gamma_pi2)
    assert np.allclose(out["s_wall"], -0.8 * H1, rtol=0, atol=1e-14)
    assert np.allclose(out["delta_f1"], -0.2 * H1, rtol=0, atol=1e-14)
    assert np.allclose(out["dF_film"], H1 * (8 + Lz), rtol=0, atol=1e-12)


def test_stiffness_and_steps_workflow():
    """Secs. III B-C: gamma = gamma_pi2 (1 + c phi^2) gives the stiffness
    constant c and kappa = gamma_pi2 (1 + 2 c) (Eqs. 23-24); the cusp gamma =
    gamma_pi2 + f_s |phi| gives f_s with the flat tension gamma_pi2 (Eq. 26,
    the flat point (pi/2, gamma_pi2) added); the step model's H1* is
    f_s / 2 - T ln(Lx) / (2 Lz) (Eq. 32) and it has no tilt at H1 = 0."""
    gamma_pi2, T, Lx, Lz = 0.9, 3.0, 32, 64
    phi = np.linspace(0.05, 0.3, 6)
    theta = math.pi / 2 - phi
    out = OW.stiffness_and_steps(theta, gamma_pi2 * (1 + 0.4 * phi ** 2), gamma_pi2, T, Lx, Lz, [0.0])
    assert abs(out["c"] - 0.4) < 1e-12 and abs(out["kappa"] - gamma_pi2 * 1.8) < 1e-12
    out = OW.stiffness_and_steps(theta, gamma_pi2 + 0.07 * phi, gamma_pi2, T, Lx, Lz, [0.0, 0.1])
    assert abs(out["f_s"] - 0.07) < 1e-12 and abs(out["gamma_flat"] - gamma_pi2) < 1e-12
    assert abs(out["h1_star"] - (0.035 - T * math.log(Lx) / (2 * Lz))) < 1e-15
    assert out["phi"][0] == 0.0 and out["phi"][1] > 0.0
    # one tilted point: the Eq. 26 line runs through it and the flat point
    out = OW.stiffness_and_steps([math.pi / 2 - 0.2], [gamma_pi2 + 0.014], gamma_pi2, T, Lx, Lz, [0.0])
    assert abs(out["f_s"] - 0.07) < 1e-12 and abs(out["gamma_flat"] - gamma_pi2) < 1e-12
