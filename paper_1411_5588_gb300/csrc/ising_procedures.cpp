// The paper's measurement procedures (Secs. II B - IV) as whole calls: each
// takes the record series of a film set, tagged by role, and composes the
// exact integer means (ising_series_mean, ising_series_energy, Eq. 17
// profiles) with the FP64 analysis calls of ising_analysis.cpp and
// ising_ti.cpp.  The arithmetic between those calls -- per-site
// normalisation, energy differences, the sign and starting point of Eq. 16's
// path -- lives here, so that a C caller needs nothing else.
#include <cmath>
#include <cstdint>
#include <vector>

#include "ising_host.h"

using namespace isg;

namespace {

bool series_ok(const ising_series& s, size_t first) {
  return s.records && s.n > first && s.Lx >= 1 && s.Ly >= 1 && s.Lz >= 1;
}

// Per-site magnetisations of layers 1 and Lx (record columns 3, 4) of a
// uniform film, averaged over records first..n-1.
int wall_means(const ising_series& s, size_t first, double* m1, double* mn) {
  const size_t stride = 5 + (size_t)s.Lx;
  const double area = (double)s.Ly * (double)s.Lz;
  double a = 0, b = 0;
  int rc = ising_series_mean(s.records, s.n, stride, 3, first, &a);
  if (!rc) rc = ising_series_mean(s.records, s.n, stride, 4, first, &b);
  if (rc) return rc;
  *m1 = a / area;
  *mn = b / area;
  return ISING_OK;
}

}  // namespace

extern "C" {

int ising_procedure_contact_angle(int k, const double* H1, int n_gl, const ising_series* inter,
                                  const ising_series* plus, const ising_series* node, size_t first, double gamma_pi2,
                                  double* theta, double* theta_young, double* delta_f1, double* gamma,
                                  double* y_plus) {
  clear_error();
  if (k < 1 || n_gl < 1 || !H1 || !inter || !plus || !node || !theta || !theta_young || !delta_f1 || !gamma ||
      !(gamma_pi2 > 0))
    return fail(ISING_EINVAL, "procedure_contact_angle: bad arguments");
  const int Lx = inter[0].Lx, Ly = inter[0].Ly, Lz = inter[0].Lz;
  std::vector<double> mbar(Lx), mp(Lx), mm(Lx), yp(Lx), m1(n_gl), mn(n_gl);
  for (int j = 0; j < k; j++) {
    const ising_series &fi = inter[j], &fp = plus[j];
    if (!series_ok(fi, first) || !series_ok(fp, first) || fi.Lx != Lx || fi.Ly != Ly || fi.Lz != Lz ||
        fp.Lx != Lx || fp.Ly != Ly || fp.Lz != Lz)
      return fail(ISING_EINVAL, "procedure_contact_angle: films of field %d differ in size or have no records", j);
    // Eq. 17 profiles, the (-) plateaus by Eq. 12, the dividing plane (Eq. 18)
    int rc = ising_layer_profile(fi.records, fi.n, Lx, Ly, Lz, first, mbar.data());
    if (!rc) rc = ising_layer_profile(fp.records, fp.n, Lx, Ly, Lz, first, mp.data());
    if (!rc) rc = ising_mirror_profile(Lx, mp.data(), mm.data());
    if (!rc) rc = ising_contact_angle(Lx, Ly, mbar.data(), mp.data(), mm.data(), 1, Lx, yp.data(), &theta[j]);
    if (rc) return rc;
    if (y_plus)
      for (int x = 0; x < Lx; x++) y_plus[(size_t)j * Lx + x] = yp[x];
    // the Young difference (Eq. 9) from the walls of the node films
    for (int i = 0; i < n_gl; i++) {
      const ising_series& f = node[(size_t)j * n_gl + i];
      if (!series_ok(f, first)) return fail(ISING_EINVAL, "procedure_contact_angle: node film %d/%d", j, i);
      rc = wall_means(f, first, &m1[i], &mn[i]);
      if (rc) return rc;
    }
    rc = ising_ti_young_difference(n_gl, H1[j], m1.data(), mn.data(), &delta_f1[j]);
    if (rc) return rc;
    // Young's angle (Eq. 8) exists only while the wall is not wet
    theta_young[j] = NAN;
    if (std::fabs(delta_f1[j]) <= gamma_pi2) {
      rc = ising_young_angle(delta_f1[j], gamma_pi2, &theta_young[j]);
      if (rc) return rc;
    }
  }
  // Eq. 16 along the measured angles, from the perpendicular interface at
  // H1 = 0 (theta = pi/2, gamma = gamma_pi2), with the acute angle's |delta_f1|
  std::vector<double> th(k + 1), df(k + 1), g(k + 1);
  th[0] = M_PI / 2;
  df[0] = 0.0;
  for (int j = 0; j < k; j++) {
    th[j + 1] = theta[j];
    df[j + 1] = std::fabs(delta_f1[j]);
  }
  const int rc = ising_gamma_of_theta(k + 1, th.data(), df.data(), gamma_pi2, g.data());
  if (rc) return rc;
  for (int j = 0; j < k; j++) gamma[j] = g[j + 1];
  return ISING_OK;
}

int ising_procedure_interface_tension(int n_sizes, const double* L, int n_beta, const double* beta,
                                      const ising_series* apbc, const ising_series* pbc, size_t first, double* dF,
                                      double* gamma_pi2, double* tau0) {
  clear_error();
  if (n_sizes < 2 || n_beta < 2 || !L || !beta || !apbc || !pbc || !dF || !gamma_pi2 || !tau0)
    return fail(ISING_EINVAL, "procedure_interface_tension: bad arguments");
  std::vector<double> dU(n_beta), F(n_beta);
  for (int s = 0; s < n_sizes; s++) {
    for (int b = 0; b < n_beta; b++) {
      const ising_series &fa = apbc[(size_t)s * n_beta + b], &fp = pbc[(size_t)s * n_beta + b];
      if (!series_ok(fa, first) || !series_ok(fp, first))
        return fail(ISING_EINVAL, "procedure_interface_tension: film %d/%d has no records", s, b);
      // <E> of Eq. 1 for the antiperiodic and the periodic film
      double ua = 0, up = 0;
      int rc = ising_series_energy(fa.records, fa.n, fa.Lx, fa.J, fa.H, fa.H1, nullptr, first, &ua);
      if (!rc) rc = ising_series_energy(fp.records, fp.n, fp.Lx, fp.J, fp.H, fp.H1, nullptr, first, &up);
      if (rc) return rc;
      dU[b] = ua - up;
    }
    // Eq. 19 from beta[0] < beta_c, where the interface free energy is 0
    const int rc = ising_ti_free_energy_beta(n_beta, beta, dU.data(), 0.0, F.data());
    if (rc) return rc;
    dF[s] = F[n_beta - 1];
  }
  return ising_fit_gamma_tau(n_sizes, L, L, dF, gamma_pi2, tau0);  // Eq. 20 with Lx = Lz = L
}

int ising_procedure_line_tension(int n_sizes, int n_gl, double H1, const ising_series* inter,
                                 const ising_series* plus, size_t first, double theta, double gamma_theta,
                                 double gamma_pi2, double* R, double* dF_film, double* s_wall, double* delta_f1,
                                 double* dtau, double* intercept) {
  clear_error();
  if (n_sizes < 2 || n_gl < 1 || !inter || !plus || !R || !dtau || !intercept)
    return fail(ISING_EINVAL, "procedure_line_tension: bad arguments");
  std::vector<double> M1(n_gl), Mn(n_gl), m1(n_gl), mn(n_gl), Lz(n_sizes);
  for (int s = 0; s < n_sizes; s++) {
    const ising_series& f0 = inter[(size_t)s * n_gl];
    for (int i = 0; i < n_gl; i++) {
      const ising_series &fi = inter[(size_t)s * n_gl + i], &fp = plus[(size_t)s * n_gl + i];
      if (!series_ok(fi, first) || !series_ok(fp, first) || fi.Lx != f0.Lx || fi.Ly != f0.Ly || fi.Lz != f0.Lz)
        return fail(ISING_EINVAL, "procedure_line_tension: film %d/%d differs in size or has no records", s, i);
      // wall totals of the film with the interface, per-site walls of the (+) film
      const size_t stride = 5 + (size_t)fi.Lx;
      int rc = ising_series_mean(fi.records, fi.n, stride, 3, first, &M1[i]);
      if (!rc) rc = ising_series_mean(fi.records, fi.n, stride, 4, first, &Mn[i]);
      if (!rc) rc = wall_means(fp, first, &m1[i], &mn[i]);
      if (rc) return rc;
    }
    double dF = 0, sw = 0, df1 = 0;
    int rc = ising_ti_surface_field(n_gl, H1, M1.data(), Mn.data(), &dF);  // F_int(H1) - F_int(0)
    if (!rc) rc = ising_ti_surface_field(n_gl, H1, m1.data(), mn.data(), &sw);  // per wall site
    if (!rc) rc = ising_ti_young_difference(n_gl, H1, m1.data(), mn.data(), &df1);
    if (!rc)
      rc = ising_line_tension_residual(dF, f0.Lx, f0.Ly, f0.Lz, theta, gamma_theta, gamma_pi2, sw, df1, &R[s]);
    if (rc) return rc;
    if (dF_film) dF_film[s] = dF;
    if (s_wall) s_wall[s] = sw;
    if (delta_f1) delta_f1[s] = df1;
    Lz[s] = f0.Lz;
  }
  return ising_line_tension_lz_scan(n_sizes, Lz.data(), R, dtau, intercept);
}

int ising_procedure_stiffness_steps(int k, const double* theta, const double* gamma, double gamma_pi2, double T,
                                    double Lx, double Lz, int n_h, const double* H1, double* c, double* kappa,
                                    double* f_s, double* gamma_flat, double* phi, double* h1_star) {
  clear_error();
  if (k < 1 || n_h < 1 || !theta || !gamma || !H1 || !c || !kappa || !f_s || !gamma_flat || !phi || !h1_star)
    return fail(ISING_EINVAL, "procedure_stiffness_steps: bad arguments");
  int rc = ising_stiffness(k, theta, gamma, gamma_pi2, c, kappa);  // Eqs. 23-24
  if (rc) return rc;
  // Eq. 26 over the flat point (pi/2, gamma_pi2) and the measured angles
  std::vector<double> th(k + 1), g(k + 1);
  th[0] = M_PI / 2;
  g[0] = gamma_pi2;
  for (int j = 0; j < k; j++) {
    th[j + 1] = theta[j];
    g[j + 1] = gamma[j];
  }
  rc = ising_step_free_energy(k + 1, th.data(), g.data(), f_s, gamma_flat);
  if (rc) return rc;
  // the single-step model at the measured f_s (Eqs. 28-32)
  for (int i = 0; i < n_h; i++) {
    double h = 0;
    rc = ising_step_model(H1[i], *f_s, T, Lx, Lz, &phi[i], &h);
    if (rc) return rc;
    if (i == 0) *h1_star = h;
  }
  return ISING_OK;
}

}  // extern "C"
